// Tall-skinny panel QR with a one-level tree: communication-avoiding QR (Eq. caqr,
// Sec. 3.1.3) with CGS2 leaves, for panels whose stacked leaf R factors fit one 1024-row
// block (P0 * B <= 1024 with B = 8 or 16 the bucketed width; at b = 16 every m <= 65536).
//
//  1. (Eq. caqr, circled 1) each of P0 CTAs factors a row block of at most RL * 256 rows by
//     CGS2, RL rows per thread in registers; its Q goes to shared memory and its b x b R to
//     the workspace.
//  2. One bounded grid barrier (cooperative launch: all CTAs are resident).
//  3. (circled 2-3) every CTA loads the P0 stacked R factors and factors the stack with the
//     same code in the same order, so each CTA holds the tree's Q without a second exchange
//     through memory. CTA 0 writes R. Each thread holds rows of one child spaced b/4 apart, so
//     in the early steps, where the upper-triangular factors' later rows are still zero, every
//     thread leaves those rows out of its arithmetic (compile-time row counts per group).
//  4. (circled 4-5) each CTA multiplies its block's Q by its b x b slice of the tree's Q and
//     stores the result: FP32 to W and, rounded to nearest even, to the product-precision
//     copy Wh.
//
// CGS2 runs in the lagged one-reduction form: one CTA-wide reduction per column gives the
// second-pass coefficients of column k against q_<k, ||a_k'||^2, the first-pass coefficients
// of column k+1 against q_<k and a_k'^T a_{k+1}, and the first-pass coefficient of column
// k+1 against q_k follows as (a_k'^T a_{k+1} - h2^T g) / R_kk. Every column is still
// orthogonalised twice; in exact arithmetic Q and R are those of CGS2. The column loop is
// unrolled in groups of four columns, so every register index is a constant and each step
// forms at most three products it does not need.
#include <mma.h>

#include "cgs2.cuh"
#include "common.cuh"
#include "kernels.cuh"

#include <stdlib.h>

namespace lls {
namespace {

constexpr int kFT = 256;            // threads per CTA
constexpr int kFW = kFT / 32;       // warps per CTA
constexpr int kStackRows = 4 * kFT;   // most stacked leaf-R rows of the tree (4 per thread)

struct FlatArgs {
    float* W; int ldw;
    void* Wh; int ldh;
    float* R; int ldr;
    int m, c0, b, P0, lowp;
    float* rbuf;            // P0 row-major B x B blocks: the leaf R factors
    unsigned* bar;          // grid barrier words (count, generation): count zero on entry
    int* err;
};

template <int B>
struct FlatSmem {
    float red[2][2][kFW][32];            // partial sums: 2 alternating buffers x 2 chunks of 32
    float tot[kFW][64];                  // per-warp copy of the CTA totals
    float Rs[B][B + 1];                  // R of the current factorization
    __align__(16) float S[B][B];         // this block's slice of the tree's Q
    int ok;
};

// CTA-wide sums of the N (<= 64) values x[] held by every thread. Returns this warp's row of
// `tot`, whose entries 0..N-1 hold the CTA totals. One barrier; `red` alternates between
// two buffers, so the next call may start writing before every warp has read this one.
template <int N, int B>
__device__ __forceinline__ const float* block_sum(const float (&x)[N], FlatSmem<B>& sm, int& parity) {
    static_assert(N >= 1 && N <= 64, "block_sum handles at most 64 values");
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    constexpr int N0 = N < 32 ? N : 32;
    constexpr int S0 = pow2ceil(N0);
    float c0[S0];
#pragma unroll
    for (int i = 0; i < S0; ++i) c0[i] = i < N0 ? x[i] : 0.f;
    sm.red[parity][0][warp][lane] = warp_transpose_reduce<S0>(c0);
    if constexpr (N > 32) {
        constexpr int S1 = pow2ceil(N - 32);
        float c1[S1];
#pragma unroll
        for (int i = 0; i < S1; ++i) c1[i] = 32 + i < N ? x[32 + i] : 0.f;
        sm.red[parity][1][warp][lane] = warp_transpose_reduce<S1>(c1);
    }
    __syncthreads();
    float t0 = 0.f;
#pragma unroll
    for (int q = 0; q < kFW; ++q) t0 += sm.red[parity][0][q][lane];
    sm.tot[warp][lane] = t0;
    if constexpr (N > 32) {
        float t1 = 0.f;
#pragma unroll
        for (int q = 0; q < kFW; ++q) t1 += sm.red[parity][1][q][lane];
        sm.tot[warp][32 + lane] = t1;
    }
    parity ^= 1;
    __syncwarp();
    return sm.tot[warp];
}

// Rows of a register block that can be nonzero up to step KMAX. A leaf (TC = 0): all R. The
// tree's stack (TC > 0): the thread holds row index (t mod TC) + TC r of one child's upper-
// triangular factor, and rows with index > KMAX are zero in columns 0..KMAX and left unchanged
// by steps 0..KMAX (their products with the current column vanish and nothing is subtracted
// from them), so only r <= KMAX / TC take part.
template <int R, int KMAX, int TC>
__host__ __device__ constexpr int active_rows() {
    return TC == 0 ? R : (KMAX / TC + 1 < R ? KMAX / TC + 1 : R);
}

// Steps K = K0 .. K0 + KG - 1 of the lagged CGS2 on the register block v (R rows per thread,
// columns 0..B-1; before step K, columns < K hold q_0..q_{K-1}, column K holds a_K after its
// first projection, the rest are raw). Afterwards column K holds q_K and column K+1 its first
// projection. Rs row j, column K accumulates R_jK (first-pass part written at step K-1,
// second-pass part added at step K).
// The KG steps of a group share one body (a runtime loop): they form the products of the
// group's widest step, with the columns not yet orthogonalised masked to zero, and pick the
// current and next columns by register selects. Sharing bodies keeps the kernel's code
// small enough for the instruction cache at a cost of at most KG - 1 extra products.
// TC: see active_rows (the tree's rows that are still zero take no part in a group's steps).
template <int B, int R, int K0, int KG, int TC>
__device__ __forceinline__ void cgs2_group(float (&v)[R][B], int b, FlatSmem<B>& sm, int& parity) {
    constexpr int NQ = K0 + KG - 1;              // q columns any step of the group may use
    constexpr int N = 2 * NQ + 2;                // h2[NQ], nn, g[NQ], c
    constexpr int RA = active_rows<R, K0 + KG - 1, TC>();   // rows that can be nonzero in the group
#pragma unroll 1
    for (int s = 0; s < KG; ++s) {
        const int K = K0 + s;
        if (K >= b) return;
        float cur[R], nx[R];
#pragma unroll
        for (int r = 0; r < RA; ++r) {
            float c = v[r][K0], d = K0 + 1 < B ? v[r][K0 + 1] : 0.f;
#pragma unroll
            for (int u = 1; u < KG; ++u) {
                c = s == u ? v[r][K0 + u] : c;
                d = s == u ? (K0 + u + 1 < B ? v[r][(K0 + u + 1) % B] : 0.f) : d;
            }
            cur[r] = c;
            nx[r] = d;
        }
        // products for columns j, j + 1 in the two halves of packed FMAs (each half is the
        // same single-rounding chain over the rows as a scalar FMA chain)
        float x[N];
#pragma unroll
        for (int j = 0; j < NQ; j += 2) {
            if (j + 1 < NQ) {
                float2 p1 = make_float2(0.f, 0.f), p2 = make_float2(0.f, 0.f);
#pragma unroll
                for (int r = 0; r < RA; ++r) {
                    const float2 vv = make_float2(v[r][j], v[r][j + 1]);
                    p1 = __ffma2_rn(vv, make_float2(cur[r], cur[r]), p1);
                    p2 = __ffma2_rn(vv, make_float2(nx[r], nx[r]), p2);
                }
                x[j] = j < K ? p1.x : 0.f;
                x[j + 1] = j + 1 < K ? p1.y : 0.f;
                x[NQ + 1 + j] = j < K ? p2.x : 0.f;
                x[NQ + 2 + j] = j + 1 < K ? p2.y : 0.f;
            } else {
                float p1 = 0.f, p2 = 0.f;
#pragma unroll
                for (int r = 0; r < RA; ++r) {
                    p1 = fmaf(v[r][j], cur[r], p1);
                    p2 = fmaf(v[r][j], nx[r], p2);
                }
                x[j] = j < K ? p1 : 0.f;
                x[NQ + 1 + j] = j < K ? p2 : 0.f;
            }
        }
        {
            float p1 = 0.f, p2 = 0.f;
#pragma unroll
            for (int r = 0; r < RA; ++r) {
                p1 = fmaf(cur[r], cur[r], p1);
                p2 = fmaf(cur[r], nx[r], p2);
            }
            x[NQ] = p1;
            x[2 * NQ + 1] = p2;
        }
        const float* t = block_sum<N, B>(x, sm, parity);

        // two interleaved chains per sum (even / odd j) halve the dependent FMA depth
        float h2[NQ > 0 ? NQ : 1], g[NQ > 0 ? NQ : 1];
#pragma unroll
        for (int j = 0; j < NQ; ++j) {
            h2[j] = t[j];                        // zero for j >= K (masked products)
            g[j] = t[NQ + 1 + j];
        }
        float2 hh2 = make_float2(0.f, 0.f), hg2 = make_float2(0.f, 0.f);   // (even j, odd j)
#pragma unroll
        for (int j = 0; j < NQ; j += 2) {
            const float2 hv = make_float2(h2[j], j + 1 < NQ ? h2[j + 1] : 0.f);
            const float2 gv = make_float2(g[j], j + 1 < NQ ? g[j + 1] : 0.f);
            hh2 = __ffma2_rn(hv, hv, hh2);
            hg2 = __ffma2_rn(hv, gv, hg2);
        }
        const float hh = hh2.x + hh2.y, hg = hg2.x + hg2.y;
        const float nn = t[NQ];
        float acc[R];
#pragma unroll
        for (int r = 0; r < RA; ++r) {
            float2 a2 = make_float2(cur[r], 0.f);   // (even j, odd j) chains
#pragma unroll
            for (int j = 0; j < NQ; j += 2)
                a2 = __ffma2_rn(make_float2(-v[r][j], j + 1 < NQ ? -v[r][j + 1] : 0.f),
                                make_float2(h2[j], j + 1 < NQ ? h2[j + 1] : 0.f), a2);
            acc[r] = a2.x + a2.y;
        }
        float normsq = nn - hh;
        if (!(normsq >= 0.25f * nn)) {   // the second pass removed much of the norm: reduce it directly
            float d[1];
            d[0] = 0.f;
#pragma unroll
            for (int r = 0; r < RA; ++r) d[0] = fmaf(acc[r], acc[r], d[0]);
            normsq = block_sum<1, B>(d, sm, parity)[0];
        }
        // R_KK and 1 / R_KK from one reciprocal square root (a few ulp; the CGS2 error bound
        // is unchanged up to the constant)
        const float ns = fmaxf(normsq, 0.f);
        const float inv = ns > 0.f ? rsqrtf(ns) : 0.f;
        const float nrm = ns * inv;
        const bool next = K + 1 < b;           // column K+1 exists (then K+1 < B)
        const float gq = next ? (t[2 * NQ + 1] - hg) * inv : 0.f;   // q_K^T a_{K+1}
        if (threadIdx.x < 32) {
            const int lane = threadIdx.x;
            if (lane < K) {
                sm.Rs[lane][K] += t[lane];
                if (next) sm.Rs[lane][K + 1] = t[NQ + 1 + lane];
            }
            if (lane == 0) {
                sm.Rs[K][K] = nrm;
                if (next) sm.Rs[K][K + 1] = gq;
            }
        }
#pragma unroll
        for (int r = 0; r < RA; ++r) {
            const float q = acc[r] * inv;
            float2 a2 = make_float2(nx[r], 0.f);    // (even j, odd j) chains
#pragma unroll
            for (int j = 0; j < NQ; j += 2)
                a2 = __ffma2_rn(make_float2(-v[r][j], j + 1 < NQ ? -v[r][j + 1] : 0.f),
                                make_float2(g[j], j + 1 < NQ ? g[j + 1] : 0.f), a2);
            const float a = fmaf(-q, gq, a2.x + a2.y);
#pragma unroll
            for (int u = 0; u < KG; ++u) {
                if (s == u) v[r][K0 + u] = q;
                if (K0 + u + 1 < B && s == u) v[r][(K0 + u + 1) % B] = a;
            }
        }
    }
}

// Steps K = K0 .. K0 + KG - 1 of modified Gram-Schmidt (Alg. 4) on the register block v:
// before step K, columns < K hold q_0..q_{K-1} and every column >= K has already had
// q_0..q_{K-1} removed. One CTA-wide reduction gives ||a_K||^2 and a_K^T a_j (j > K); then
// R_KK = ||a_K||, q_K = a_K / R_KK, R_Kj = a_K^T a_j / R_KK (= q_K^T a_j) and
// a_j -= q_K R_Kj. Products for columns j <= K are masked to zero, so the shared group body
// leaves them untouched. TC as in cgs2_group.
template <int B, int R, int K0, int KG, int TC>
__device__ __forceinline__ void mgs_group(float (&v)[R][B], int b, FlatSmem<B>& sm, int& parity) {
    constexpr int RA = active_rows<R, K0 + KG - 1, TC>();
    constexpr int N = B - K0;                    // ||a_K||^2, then a_K^T a_j for j = K0+1 .. B-1
#pragma unroll 1
    for (int s = 0; s < KG; ++s) {
        const int K = K0 + s;
        if (K >= b) return;
        float cur[R];
#pragma unroll
        for (int r = 0; r < RA; ++r) {
            float c = v[r][K0];
#pragma unroll
            for (int u = 1; u < KG; ++u) c = s == u ? v[r][K0 + u] : c;
            cur[r] = c;
        }
        float x[N];
        {
            float p = 0.f;
#pragma unroll
            for (int r = 0; r < RA; ++r) p = fmaf(cur[r], cur[r], p);
            x[0] = p;
        }
#pragma unroll
        for (int i = 1; i < N; ++i) {
            const int j = K0 + i;
            float p = 0.f;
#pragma unroll
            for (int r = 0; r < RA; ++r) p = fmaf(v[r][j], cur[r], p);
            x[i] = j > K ? p : 0.f;
        }
        const float* t = block_sum<N, B>(x, sm, parity);
        const float ns = fmaxf(t[0], 0.f);
        const float inv = ns > 0.f ? rsqrtf(ns) : 0.f;
        const float nrm = ns * inv;
        float rk[N];                             // R_Kj for j = K0 + i (zero for j <= K)
        rk[0] = 0.f;
#pragma unroll
        for (int i = 1; i < N; ++i) rk[i] = t[i] * inv;
        if (threadIdx.x < 32) {
            const int lane = threadIdx.x;
            if (lane == 0) sm.Rs[K][K] = nrm;
            if (lane > K && lane < b) sm.Rs[K][lane] = t[lane - K0] * inv;
        }
#pragma unroll
        for (int r = 0; r < RA; ++r) {
            const float q = cur[r] * inv;
#pragma unroll
            for (int i = 1; i < N; ++i) v[r][K0 + i] = fmaf(-q, rk[i], v[r][K0 + i]);
#pragma unroll
            for (int u = 0; u < KG; ++u)
                if (s == u) v[r][K0 + u] = q;
        }
    }
}

template <int B, int R, int K0, int TC>
struct MgsFlat {
    static constexpr int KG = 4;
    static __device__ __forceinline__ void run(float (&v)[R][B], int b, FlatSmem<B>& sm, int& parity) {
        if (K0 >= b) return;
        mgs_group<B, R, K0, KG, TC>(v, b, sm, parity);
        MgsFlat<B, R, K0 + KG, TC>::run(v, b, sm, parity);
    }
};
template <int B, int R, int TC>
struct MgsFlat<B, R, B, TC> {
    static __device__ __forceinline__ void run(float (&)[R][B], int, FlatSmem<B>&, int&) {}
};

// CGS2 steps per shared group body, for blocks of 2 rows per thread (LEAF: the 512-row leaves and
// the 512-row tree stack) and of 4 rows per thread (TREE: the 1024-row leaves and stack). Fewer steps per body mean fewer masked products but more code for the
// instruction cache; on the 32768 x 16 panel two steps per body measured fastest (block
// 75.8 us, against 77.8 with four and 88.4 with one).
#ifndef LLS_CGS_GROUP_LEAF
#define LLS_CGS_GROUP_LEAF 2
#endif
#ifndef LLS_CGS_GROUP_TREE
#define LLS_CGS_GROUP_TREE 2
#endif
template <int R>
constexpr int cgs_group() { return R <= 2 ? LLS_CGS_GROUP_LEAF : LLS_CGS_GROUP_TREE; }

template <int B, int R, int K0, int TC>
struct Cgs2Flat {
    static constexpr int KG = cgs_group<R>() < B ? cgs_group<R>() : B;
    static __device__ __forceinline__ void run(float (&v)[R][B], int b, FlatSmem<B>& sm, int& parity) {
        if (K0 >= b) return;
        cgs2_group<B, R, K0, KG, TC>(v, b, sm, parity);
        Cgs2Flat<B, R, K0 + KG, TC>::run(v, b, sm, parity);
    }
};
template <int B, int R, int TC>
struct Cgs2Flat<B, R, B, TC> {
    static __device__ __forceinline__ void run(float (&)[R][B], int, FlatSmem<B>&, int&) {}
};

// The factorization of a register block: CGS2 (default) or MGS (Alg. 4). TC = 0: a leaf (rows
// of the panel); TC > 0: the tree's stack in the layout of panel_body (TC threads per child).
template <bool MGS, int B, int R, int TC = 0>
__device__ __forceinline__ void leaf_qr(float (&v)[R][B], int b, FlatSmem<B>& sm, int& parity) {
    if constexpr (MGS) MgsFlat<B, R, 0, TC>::run(v, b, sm, parity);
    else Cgs2Flat<B, R, 0, TC>::run(v, b, sm, parity);
}

__device__ __forceinline__ void flat_leaf_range(int m, int P0, int i, int& s, int& e) {
    const int base = m / P0, extra = m % P0;
    s = i * base + min(i, extra);
    e = s + base + (i < extra ? 1 : 0);
}

#if LLS_DEBUG
// Planted faults for the tests of the debug build: 1 = every store of Q is addressed one panel
// height too low (the index checks reject it); 2 = the leaf-to-tree grid barrier waits for one
// CTA more than the grid holds (the bounded wait gives up).
__device__ int g_debug_inject;
#endif

__device__ __forceinline__ void flat_store_q(const FlatArgs& a, int row, int j, float q) {
#if LLS_DEBUG
    if (g_debug_inject == 1) row += a.m;
#endif
    if (!LLS_INB(row >= 0 && row < a.m && j >= 0 && j < a.b)) return;
    a.W[(size_t)row + (size_t)(a.c0 + j) * a.ldw] = q;
    const size_t h = (size_t)row + (size_t)(a.c0 + j) * a.ldh;
    if (a.lowp == 0) reinterpret_cast<__half*>(a.Wh)[h] = __float2half_rn(q);
    else if (a.lowp == 1) reinterpret_cast<__nv_bfloat16*>(a.Wh)[h] = __float2bfloat16_rn(q);
}

template <int B>
__device__ __forceinline__ void flat_write_r(const FlatArgs& a, const FlatSmem<B>& sm) {
    for (int i = threadIdx.x; i < a.b * a.b; i += kFT) {
        const int r = i % a.b, c = i / a.b;
        if (!LLS_INB(r < B && c < B && a.c0 + r < a.ldr)) continue;
        a.R[(size_t)(a.c0 + r) + (size_t)(a.c0 + c) * a.ldr] = r <= c ? sm.Rs[r][c] : 0.f;
    }
}

// The panel of columns [a.c0, a.c0 + b), this CTA's rows [s, s + rows) of which are in v:
// leaf factorization, the one-level tree and the reconstruction. Q goes to W and Wh, R to R
// (CTA 0). On return v holds this CTA's rows of Q (zero beyond `rows`). Returns false if a
// bounded grid barrier gave up (the error word is set).
template <int B, int RL, int RR, bool MGS>
__device__ __forceinline__ bool panel_body(const FlatArgs& a, float (&v)[RL][B], FlatSmem<B>& sm, float* Ql, int& parity,
                           int s, int rows) {
    const int t = threadIdx.x, b = a.b;
    for (int i = t; i < B * (B + 1); i += kFT) (&sm.Rs[0][0])[i] = 0.f;
    for (int i = t; i < B * B; i += kFT) (&sm.S[0][0])[i] = 0.f;
    __syncthreads();
    leaf_qr<MGS, B, RL>(v, b, sm, parity);
    __syncthreads();

    if (a.P0 == 1) {   // the block is the whole panel: Q and R are final
#pragma unroll
        for (int r = 0; r < RL; ++r) {
            const int lr = t + r * kFT;
            if (lr >= rows) continue;
#pragma unroll
            for (int j = 0; j < B; ++j)
                if (j < b) flat_store_q(a, s + lr, j, v[r][j]);
        }
        flat_write_r<B>(a, sm);
        __syncthreads();
        return true;
    }

    // leaf Q to shared memory, leaf R to the workspace
#pragma unroll
    for (int r = 0; r < RL; ++r)
#pragma unroll
        for (int j = 0; j < B; ++j) Ql[(t + r * kFT) * (B + 1) + j] = v[r][j];
    float* rb = a.rbuf + (size_t)blockIdx.x * (B * B);
    if (LLS_INB((int)blockIdx.x < a.P0))
        for (int i = t; i < B * B; i += kFT) rb[i] = sm.Rs[i / B][i % B];
    // no fence per thread: the grid barrier's CTA barrier followed by its thread 0's fence
    // releases every thread's stores before the arrival
    __syncthreads();
    for (int i = t; i < B * (B + 1); i += kFT) (&sm.Rs[0][0])[i] = 0.f;

    // bounded grid barrier: every leaf R is in the workspace
#if LLS_DEBUG
    const unsigned expect = a.P0 + (g_debug_inject == 2 ? 1 : 0);
#else
    const unsigned expect = a.P0;
#endif
    if (!grid_barrier(a.bar, expect, a.err)) return false;

    // the stacked R factors: TC = B / 4 threads per child, thread t holding rows
    // (t mod TC) + TC r (r < RR) of child t / TC, so that in step K only the rows r <= K / TC can
    // be nonzero (upper-triangular factors) and every thread takes part in the same share
    constexpr int TC = B / 4;
    static_assert(RR * TC == B && kFT / TC * B == kStackRows, "tree layout: 4 rows of each child per thread");
    const int child = t / TC, rsub = t % TC;
    float vr[RR][B];
    {
        const bool live = child < a.P0 && LLS_INB(child >= 0);
#pragma unroll
        for (int r = 0; r < RR; ++r) {
            const int rr = rsub + TC * r;
            const float4* src = reinterpret_cast<const float4*>(a.rbuf + (size_t)child * (B * B) + rr * B);
#pragma unroll
            for (int j4 = 0; j4 < B / 4; ++j4) {
                const float4 q = (live && rr < b) ? __ldcg(src + j4) : make_float4(0.f, 0.f, 0.f, 0.f);
                vr[r][4 * j4 + 0] = q.x; vr[r][4 * j4 + 1] = q.y; vr[r][4 * j4 + 2] = q.z; vr[r][4 * j4 + 3] = q.w;
            }
        }
    }
    leaf_qr<MGS, B, RR, TC>(vr, b, sm, parity);
    // this block's b x b slice of the tree's Q: the rows of child blockIdx.x
    if (child == (int)blockIdx.x) {
#pragma unroll
        for (int r = 0; r < RR; ++r) {
            const int rr = rsub + TC * r;
            if (rr < b)
#pragma unroll
                for (int j = 0; j < B; ++j) sm.S[rr][j] = vr[r][j];
        }
    }
    __syncthreads();
    if (blockIdx.x == 0) flat_write_r<B>(a, sm);
    // Q = Q_leaf * S
#pragma unroll
    for (int r = 0; r < RL; ++r) {
        const int lr = t + r * kFT;
        if (lr >= rows) {
#pragma unroll
            for (int j = 0; j < B; ++j) v[r][j] = 0.f;
            continue;
        }
        float q[B];
#pragma unroll
        for (int k = 0; k < B; ++k) q[k] = Ql[lr * (B + 1) + k];
        float o[B];
#pragma unroll
        for (int j = 0; j < B; ++j) o[j] = 0.f;
#pragma unroll
        for (int k = 0; k < B; ++k) {
            const float4* Sk = reinterpret_cast<const float4*>(&sm.S[k][0]);
            const float2 qk = make_float2(q[k], q[k]);
#pragma unroll
            for (int j4 = 0; j4 < B / 4; ++j4) {
                const float4 s4 = Sk[j4];
                float2 lo = __ffma2_rn(qk, make_float2(s4.x, s4.y), make_float2(o[4 * j4 + 0], o[4 * j4 + 1]));
                float2 hi = __ffma2_rn(qk, make_float2(s4.z, s4.w), make_float2(o[4 * j4 + 2], o[4 * j4 + 3]));
                o[4 * j4 + 0] = lo.x; o[4 * j4 + 1] = lo.y; o[4 * j4 + 2] = hi.x; o[4 * j4 + 3] = hi.y;
            }
        }
#pragma unroll
        for (int j = 0; j < B; ++j) {
            v[r][j] = o[j];
            if (j < b) flat_store_q(a, s + lr, j, o[j]);
        }
    }
    __syncthreads();   // Ql, S and Rs are free again
    return true;
}

template <int B, int RL>
__device__ __forceinline__ void load_rows(const FlatArgs& a, int c0, float (&v)[RL][B], int s, int rows, int ncol) {
#pragma unroll
    for (int r = 0; r < RL; ++r) {
        const int lr = threadIdx.x + r * kFT;
#pragma unroll
        for (int j = 0; j < B; ++j)
            v[r][j] = (lr < rows && j < ncol && LLS_INB(s + lr >= 0 && s + lr < a.m))
                          ? a.W[(size_t)(s + lr) + (size_t)(c0 + j) * a.ldw] : 0.f;
    }
}

template <int B, int RL, int RR, bool MGS>
__global__ void __launch_bounds__(kFT, 1) panel_flat_kernel(FlatArgs a) {
    extern __shared__ __align__(128) unsigned char flat_smem[];
    FlatSmem<B>& sm = *reinterpret_cast<FlatSmem<B>*>(flat_smem);
    float* Ql = reinterpret_cast<float*>(flat_smem + sizeof(FlatSmem<B>));   // [RL * kFT][B + 1]
    int parity = 0;
    int s, e;
    flat_leaf_range(a.m, a.P0, blockIdx.x, s, e);
    float v[RL][B];
    load_rows<B, RL>(a, a.c0, v, s, e - s, a.b);
    panel_body<B, RL, RR, MGS>(a, v, sm, Ql, parity, s, e - s);
}

// ---- a block of two panels and the recursion node between them, in one launch ----------
//
// At the lowest internal nodes of the recursion (w = w1 + w2 with w1 = the panel width) the
// left panel, the node's two products and the right panel run as one cooperative launch; the
// CTAs keep the same rows throughout, so A2 goes from its load through the update into the
// second panel in registers:
//   1. panel of columns [c0, c0 + w1) (panel_body): Q1 rows in registers, Q1l = round(Q1) in
//      shared memory (the copy the panel also stores to Wh);
//   2. FP16: e_j from the column maxima of |A2| over the CTA's own rows; A2l = round(A2 2^e_j);
//   3. the CTA's partial Q1l^T A2l (warp MMAs, FP32 accumulation, fixed-order warp sum),
//      times 2^-e_j -> grid barrier -> every CTA sums the P0 partials in the same fixed order,
//      so all hold the same R12 (CTA 0 writes it to R), f_j and R12l = round(R12 2^f_j);
//   4. A2 -= (Q1l R12l) 2^-f_j for the CTA's rows (warp MMAs, FP32), in registers;
//   5. panel of columns [c0 + w1, c0 + w1 + w2) on the updated rows.
// The rounding points are those of the separate kernels (Alg. 2 with the column scaling of
// Sec. 3.1.2); only the order of the FP32 accumulations differs. The separate kernels scale
// column j by one exponent e_j from its maximum over all rows; here each CTA takes the
// exponent of its own rows' maximum, which is never smaller. Scaling by a power of two
// commutes with rounding to FP16 and with the FP32 accumulation while the values stay
// normal, so every partial times 2^-e_j is the same number either way (where the common
// exponent would leave a value among FP16's subnormals the CTA's exponent keeps more of
// it), and the grid barrier that a common exponent needs is saved.

constexpr int kBlkLdK = 8;          // padding (halves) of the K-contiguous operand rows
constexpr int kUsLd = 20;           // row stride (floats) of the update products

constexpr int kBlockMaxP0 = kStackRows / 16;   // CTAs of a one-level panel of width 16

struct BlockArgs {
    FlatArgs p1, p2;                // the two panels
    float* part;                    // P0 x 256 projection partials
    int w1, w2, kind;               // kind: 1 FP16 column scaling, 0 none (BF16)
};

template <typename TL, int RL>
struct BlockSmem {
    __align__(32) TL Qs[16][RL * kFT + kBlkLdK];   // Q1l: Qs[i][row]
    __align__(32) TL As[16][RL * kFT + kBlkLdK];   // A2l: As[j][row]
    __align__(32) TL Rl[16][16];                   // R12l column-major: Rl[j][i]
    __align__(32) float wp[kFW][256];              // per-warp projection partials (column-major)
    __align__(32) float us[kFW][32][kUsLd];        // per-warp update products, row-major
    float r12[16][17];                             // R12: r12[j][i]
    float red[kFW][16];                            // per-warp column maxima
    float sc[16], einv[16], fpos[16], fneg[16];    // 2^e_j, 2^-e_j, 2^f_j, 2^-f_j
};

template <int RL>
constexpr size_t block_ql_off() { return (sizeof(FlatSmem<16>) + 127) / 128 * 128; }
template <typename TL, int RL>
constexpr size_t block_node_off() {
    return (block_ql_off<RL>() + sizeof(float) * RL * kFT * 17 + 127) / 128 * 128;
}
template <typename TL, int RL>
constexpr size_t block_smem_bytes() { return block_node_off<TL, RL>() + sizeof(BlockSmem<TL, RL>); }

// Steps 1 (Q1l), 2, 3 and 4 of the block for this CTA's rows: on entry v holds the rows of Q1,
// on return the rows of the updated A2. False if a grid barrier gave up.
template <typename TL, int RL>
__device__ __forceinline__ bool block_node(const BlockArgs& a, float (&v)[RL][16], BlockSmem<TL, RL>& bs,
                                           int s, int rows) {
    using namespace nvcuda;
    constexpr int kLd = RL * kFT + kBlkLdK;
    const int t = threadIdx.x, lane = t & 31, warp = t >> 5;
    const int P0 = a.p1.P0, w1 = a.w1, w2 = a.w2;
#pragma unroll
    for (int r = 0; r < RL; ++r)
#pragma unroll
        for (int i = 0; i < 16; ++i) bs.Qs[i][t + r * kFT] = LowPrec<TL>::from_float(v[r][i]);

    // 2. A2 rows; FP16 column scaling from the column maxima over this CTA's rows
    load_rows<16, RL>(a.p1, a.p1.c0 + w1, v, s, rows, w2);
    if (a.kind != 0) {
        float mx[16];
#pragma unroll
        for (int j = 0; j < 16; ++j) {
            float x = 0.f;
#pragma unroll
            for (int r = 0; r < RL; ++r) x = fmaxf(x, fabsf(v[r][j]));
            mx[j] = x;
        }
        const float wm = warp_transpose_max<16>(mx);
        if (lane < 16) bs.red[warp][lane] = wm;
        __syncthreads();
        if (t < 16) {
            float x = 0.f;
#pragma unroll
            for (int q = 0; q < kFW; ++q) x = fmaxf(x, bs.red[q][t]);
            const int ej = scale_exponent(1, t < w2 ? x : 0.f);
            bs.sc[t] = pow2f(ej);
            bs.einv[t] = pow2f(-ej);
        }
    } else if (t < 16) {
        bs.sc[t] = 1.f;
        bs.einv[t] = 1.f;
    }
    __syncthreads();
#pragma unroll
    for (int r = 0; r < RL; ++r)
#pragma unroll
        for (int j = 0; j < 16; ++j) bs.As[j][t + r * kFT] = LowPrec<TL>::from_float(v[r][j] * bs.sc[j]);
    __syncwarp();   // a warp's MMA steps read only the rows its own lanes wrote

    // 3. projection partials: warp w takes the 32-row slices w of every 256-row group
    {
        wmma::fragment<wmma::accumulator, 16, 16, 16, float> acc;
        wmma::fill_fragment(acc, 0.f);
#pragma unroll
        for (int r = 0; r < RL; ++r)
#pragma unroll
            for (int h = 0; h < 2; ++h) {
                const int k0 = r * kFT + warp * 32 + h * 16;
                wmma::fragment<wmma::matrix_a, 16, 16, 16, TL, wmma::row_major> fa;
                wmma::fragment<wmma::matrix_b, 16, 16, 16, TL, wmma::col_major> fb;
                wmma::load_matrix_sync(fa, &bs.Qs[0][k0], kLd);
                wmma::load_matrix_sync(fb, &bs.As[0][k0], kLd);
                wmma::mma_sync(acc, fa, fb, acc);
            }
        wmma::store_matrix_sync(&bs.wp[warp][0], acc, 16, wmma::mem_col_major);
    }
    __syncthreads();
    {
        float x = 0.f;
#pragma unroll
        for (int q = 0; q < kFW; ++q) x += bs.wp[q][t];   // entry (t mod 16, t / 16)
        x *= bs.einv[t >> 4];                              // exact: a power of two
        if (LLS_INB((int)blockIdx.x < kBlockMaxP0 && t < 256)) a.part[(size_t)blockIdx.x * 256 + t] = x;
    }
    if (!grid_barrier(a.p1.bar, P0, a.p1.err)) return false;
    {
        // entry t summed over the P0 partials in a fixed order; all loads are issued first
        const float* p = a.part + t;
        float x[kBlockMaxP0];
#pragma unroll
        for (int c = 0; c < kBlockMaxP0; ++c) x[c] = c < P0 ? __ldcg(p + (size_t)c * 256) : 0.f;
        float acc[8];
#pragma unroll
        for (int u = 0; u < 8; ++u) {
            float s8 = 0.f;
#pragma unroll
            for (int c = u; c < kBlockMaxP0; c += 8) s8 += x[c];
            acc[u] = s8;
        }
        const float tot = ((acc[0] + acc[1]) + (acc[2] + acc[3])) + ((acc[4] + acc[5]) + (acc[6] + acc[7]));
        const int i = t & 15, j = t >> 4;
        const bool live = i < w1 && j < w2;
        const float r12 = live ? tot : 0.f;
        bs.r12[j][i] = r12;
        if (blockIdx.x == 0 && live && LLS_INB(a.p1.c0 + i < a.p1.ldr))
            a.p1.R[(size_t)(a.p1.c0 + i) + (size_t)(a.p1.c0 + w1 + j) * a.p1.ldr] = r12;
    }
    __syncthreads();
    if (t < 16) {
        float mx = 0.f;
#pragma unroll
        for (int i = 0; i < 16; ++i) mx = fmaxf(mx, fabsf(bs.r12[t][i]));
        const int fj = scale_exponent(a.kind, mx);
        bs.fpos[t] = pow2f(fj);
        bs.fneg[t] = pow2f(-fj);
    }
    __syncthreads();
    bs.Rl[t >> 4][t & 15] = LowPrec<TL>::from_float(bs.r12[t >> 4][t & 15] * bs.fpos[t >> 4]);
    __syncthreads();

    // 4. A2 -= (Q1l R12l) 2^-f_j on this warp's rows
    {
        float* us = &bs.us[warp][0][0];
        wmma::fragment<wmma::matrix_b, 16, 16, 16, TL, wmma::col_major> fb;
        wmma::load_matrix_sync(fb, &bs.Rl[0][0], 16);
        float fneg[16];
#pragma unroll
        for (int j = 0; j < 16; ++j) fneg[j] = bs.fneg[j];
#pragma unroll
        for (int r = 0; r < RL; ++r) {
#pragma unroll
            for (int h = 0; h < 2; ++h) {
                wmma::fragment<wmma::matrix_a, 16, 16, 16, TL, wmma::col_major> fa;
                wmma::load_matrix_sync(fa, &bs.Qs[0][r * kFT + warp * 32 + h * 16], kLd);
                wmma::fragment<wmma::accumulator, 16, 16, 16, float> acc;
                wmma::fill_fragment(acc, 0.f);
                wmma::mma_sync(acc, fa, fb, acc);
                wmma::store_matrix_sync(us + h * 16 * kUsLd, acc, kUsLd, wmma::mem_row_major);
            }
            __syncwarp();
            const float4* u4 = reinterpret_cast<const float4*>(us + lane * kUsLd);
#pragma unroll
            for (int j4 = 0; j4 < 4; ++j4) {
                const float4 u = u4[j4];
                v[r][4 * j4 + 0] = fmaf(-u.x, fneg[4 * j4 + 0], v[r][4 * j4 + 0]);
                v[r][4 * j4 + 1] = fmaf(-u.y, fneg[4 * j4 + 1], v[r][4 * j4 + 1]);
                v[r][4 * j4 + 2] = fmaf(-u.z, fneg[4 * j4 + 2], v[r][4 * j4 + 2]);
                v[r][4 * j4 + 3] = fmaf(-u.w, fneg[4 * j4 + 3], v[r][4 * j4 + 3]);
            }
            __syncwarp();
        }
    }

    return true;
}

template <typename TL, int RL, int RR>
__global__ void __launch_bounds__(kFT, 1) block_fused_kernel(BlockArgs a) {
    extern __shared__ __align__(128) unsigned char flat_smem[];
    FlatSmem<16>& sm = *reinterpret_cast<FlatSmem<16>*>(flat_smem);
    float* Ql = reinterpret_cast<float*>(flat_smem + block_ql_off<RL>());
    BlockSmem<TL, RL>& bs = *reinterpret_cast<BlockSmem<TL, RL>*>(flat_smem + block_node_off<TL, RL>());
    int parity = 0, s, e;
    flat_leaf_range(a.p1.m, a.p1.P0, blockIdx.x, s, e);
    const int rows = e - s;
    float v[RL][16];
    load_rows<16, RL>(a.p1, a.p1.c0, v, s, rows, a.w1);
    // the two panels share one copy of the panel code (a two-trip loop), which keeps the
    // kernel within the instruction cache
    FlatArgs pa = a.p1;
#pragma unroll 1
    for (int pass = 0;; ++pass) {
        if (!panel_body<16, RL, RR, false>(pa, v, sm, Ql, parity, s, rows)) return;   // 1. / 5.
        if (pass == 1) break;
        if (!block_node<TL, RL>(a, v, bs, s, rows)) return;                      // 1. - 4.
        pa = a.p2;
    }
}

template <int B, int RL>
constexpr size_t flat_smem_bytes() {
    return sizeof(FlatSmem<B>) + (size_t)RL * kFT * (B + 1) * sizeof(float);
}

// Per device: the dynamic shared memory opt-in and the co-resident CTA capacity.
template <int B, int RL, int RR, bool MGS>
static int flat_prepare(int& capacity) {
    constexpr int kMaxDev = 64;
    static int cap[kMaxDev];
    static bool done[kMaxDev];
    int dev = 0;
    LLS_CUDA_TRY(cudaGetDevice(&dev));
    if (dev < 0 || dev >= kMaxDev) return LLS_ERR_UNSUPPORTED;
    if (!done[dev]) {
        const size_t smem = flat_smem_bytes<B, RL>();
        LLS_CUDA_TRY(cudaFuncSetAttribute(panel_flat_kernel<B, RL, RR, MGS>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                          (int)smem));
        int sms = 0, per = 0;
        LLS_CUDA_TRY(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
        LLS_CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, panel_flat_kernel<B, RL, RR, MGS>, kFT, smem));
        cap[dev] = sms * per;
        done[dev] = true;
    }
    capacity = cap[dev];
    return LLS_OK;
}

template <int B, int RL, int RR, bool MGS>
static int launch_flat(FlatArgs& a, cudaStream_t st) {
    int cap = 0;
    LLS_TRY((flat_prepare<B, RL, RR, MGS>(cap)));
    if (a.P0 > cap) return LLS_ERR_UNSUPPORTED;
    const size_t smem = flat_smem_bytes<B, RL>();
    if (a.P0 == 1) {
        panel_flat_kernel<B, RL, RR, MGS><<<1, kFT, smem, st>>>(a);
    } else {
        void* args[] = {&a};
        LLS_CUDA_TRY(cudaLaunchCooperativeKernel((void*)panel_flat_kernel<B, RL, RR, MGS>, dim3(a.P0), dim3(kFT), args,
                                                 smem, st));
    }
    LLS_LAUNCH_CHECK("panel_flat", st);
    return LLS_OK;
}

template <typename TL, int RL, int RR>
static int launch_block(BlockArgs& a, cudaStream_t st) {
    static_assert(block_smem_bytes<TL, RL>() <= 227 * 1024, "shared memory of one CTA");
    constexpr int kMaxDev = 64;
    static int cap[kMaxDev];
    static bool done[kMaxDev];
    int dev = 0;
    LLS_CUDA_TRY(cudaGetDevice(&dev));
    if (dev < 0 || dev >= kMaxDev) return LLS_ERR_UNSUPPORTED;
    const size_t smem = block_smem_bytes<TL, RL>();
    if (!done[dev]) {
        LLS_CUDA_TRY(cudaFuncSetAttribute(block_fused_kernel<TL, RL, RR>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                          (int)smem));
        int sms = 0, per = 0;
        LLS_CUDA_TRY(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
        LLS_CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, block_fused_kernel<TL, RL, RR>, kFT, smem));
        cap[dev] = sms * per;
        done[dev] = true;
    }
    if (a.p1.P0 > cap[dev]) return LLS_ERR_UNSUPPORTED;
    if (a.p1.P0 == 1) {
        block_fused_kernel<TL, RL, RR><<<1, kFT, smem, st>>>(a);
    } else {
        void* args[] = {&a};
        LLS_CUDA_TRY(cudaLaunchCooperativeKernel((void*)block_fused_kernel<TL, RL, RR>, dim3(a.p1.P0), dim3(kFT), args,
                                                 smem, st));
    }
    LLS_LAUNCH_CHECK("block_fused", st);
    return LLS_OK;
}

// Leaf shape of a one-level panel of m rows and bucketed width bw: rows per thread of the
// leaves (rl), number of CTAs (P0) and stacked rows per thread of the tree (rr); false when the
// stacked leaf R factors would not fit one 1024-row block. 512-row leaves are taken wherever
// their stack fits: 1024-row leaves with a 512-row stack (two rows per thread in the tree) were
// measured slower at 32768 x 16 (panel 33.2 us against 30.2).
static bool flat_long_leaves() {
    static const bool v = [] {
        const char* s = getenv("LLS_FLAT");
        return s && s[0] == 'l';   // LLS_FLAT=long: 1024-row leaves wherever the stack fits
    }();
    return v;
}

static bool flat_shape(int m, int bw, int& rl, int& P0, int& rr) {
    const int p2 = ceil_div(m, 2 * kFT), p4 = ceil_div(m, 4 * kFT);
    rr = 4;
    if (m <= 2 * kFT) { rl = 2; P0 = 1; }
    else if (m <= 4 * kFT) { rl = 4; P0 = 1; }
    else if (flat_long_leaves() && p4 * bw <= kStackRows) { rl = 4; P0 = p4; }
    else if (p2 * bw <= kStackRows) { rl = 2; P0 = p2; }
    else if (p4 * bw <= kStackRows) { rl = 4; P0 = p4; }
    else return false;
    return true;
}

template <int B, bool MGS>
static int launch_flat_shape(FlatArgs& a, int rl, int rr, cudaStream_t st) {
    (void)rr;
    return rl == 2 ? launch_flat<B, 2, 4, MGS>(a, st) : launch_flat<B, 4, 4, MGS>(a, st);
}

template <typename TL>
static int launch_block_shape(BlockArgs& a, int rl, int rr, cudaStream_t st) {
    (void)rr;
    return rl == 2 ? launch_block<TL, 2, 4>(a, st) : launch_block<TL, 4, 4>(a, st);
}

bool flat_disabled() {
    static const bool off = [] {
        const char* s = getenv("LLS_PANEL");
        return s && s[0] == 't';   // LLS_PANEL=tree: always the multi-level kernel
    }();
    return off;
}

}  // namespace

int panel_debug_inject(int mode) {
#if LLS_DEBUG
    const int v = mode;
    LLS_CUDA_TRY(cudaMemcpyToSymbol(g_debug_inject, &v, sizeof(v)));
    return LLS_OK;
#else
    (void)mode;
    return LLS_ERR_UNSUPPORTED;
#endif
}

// Returns LLS_ERR_UNSUPPORTED (nothing launched) when the panel needs a deeper tree.
int panel_flat_qr(const PanelCall& c, cudaStream_t st) {
    if (flat_disabled() || c.b < 1 || c.b > 16) return LLS_ERR_UNSUPPORTED;
    FlatArgs a;
    a.W = c.W; a.ldw = c.ldw; a.Wh = c.Wh; a.ldh = c.ldh; a.R = c.R; a.ldr = c.ldr;
    a.m = c.m; a.c0 = c.c0; a.b = c.b; a.lowp = c.lowp;
    a.rbuf = c.rbuf; a.bar = c.cnt + kFlatBarWord; a.err = c.err;
    const int bw = c.b <= 8 ? 8 : 16;   // the stack holds TPR * 4 children of B rows each
    int rl, rr;
    if (!flat_shape(c.m, bw, rl, a.P0, rr)) return LLS_ERR_UNSUPPORTED;
    if (c.leaf == 1)
        return c.b <= 8 ? launch_flat_shape<8, true>(a, rl, rr, st) : launch_flat_shape<16, true>(a, rl, rr, st);
    return c.b <= 8 ? launch_flat_shape<8, false>(a, rl, rr, st) : launch_flat_shape<16, false>(a, rl, rr, st);
}

size_t block_fused_part_floats() { return (size_t)kBlockMaxP0 * 256; }

bool block_fused_supported(const BlockCall& c) {
    if (flat_disabled() || (c.lowp != 0 && c.lowp != 1)) return false;
    if (c.w1 <= 8 || c.w1 > 16 || c.w2 < 1 || c.w2 > c.w1) return false;
    int rl, P0, rr;
    return flat_shape(c.m, 16, rl, P0, rr) && P0 <= kBlockMaxP0 && (size_t)P0 * 256 <= c.part_floats;
}

int block_fused_qr(const BlockCall& c, cudaStream_t st) {
    if (!block_fused_supported(c)) return LLS_ERR_UNSUPPORTED;
    BlockArgs a;
    FlatArgs& p = a.p1;
    p.W = c.W; p.ldw = c.ldw; p.Wh = c.Wh; p.ldh = c.ldh; p.R = c.R; p.ldr = c.ldr;
    p.m = c.m; p.c0 = c.c0; p.b = c.w1; p.lowp = c.lowp;
    p.rbuf = c.rbuf; p.bar = c.cnt + kFlatBarWord; p.err = c.err;
    int rl, rr;
    flat_shape(c.m, 16, rl, p.P0, rr);
    a.p2 = p;
    a.p2.c0 = c.c0 + c.w1;
    a.p2.b = c.w2;
    a.part = c.part; a.w1 = c.w1; a.w2 = c.w2; a.kind = c.lowp == 0 ? 1 : 0;
    if (c.lowp == 0) return launch_block_shape<__half>(a, rl, rr, st);
    return launch_block_shape<__nv_bfloat16>(a, rl, rr, st);
}

}  // namespace lls
