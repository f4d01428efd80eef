// Batched least squares: many independent uneven problems in one persistent launch.
//
// Each CTA takes whole problems from a device work queue (ordered by estimated cost,
// largest first) and runs the complete hot path for each one on its own SM:
//   copy A -> W; recursive Gram-Schmidt QR (Alg. 2) with 16-column panels; the panel is the
//   communication-avoiding QR of Eq. caqr over 1024-row blocks processed one after another
//   (CGS2 on register-resident blocks, the same routine as the multi-CTA panel); the two
//   products of each recursion step run on the tensor cores (FP16/BF16 inputs, FP32
//   accumulation, warp-level MMA fragments) with the power-of-two column scaling; then
//   R^{-1} (Eq. recqr block inverse); then R-preconditioned CGLS (Alg. 5) with compensated
//   (double-float) products and block-level reductions; finally a fresh residual check.
// No grid-wide synchronisation: a CTA never waits for another one.
#include <mma.h>

#include <algorithm>
#include <numeric>
#include <vector>

#include "cgs2.cuh"
#include "common.cuh"
#include "kernels.cuh"

namespace lls {

using namespace nvcuda;

constexpr int kBPw = 16;           // panel width of the batched path
constexpr int kBMaxBlocks = 8;     // 1024-row blocks per panel (m <= 8192)
constexpr int kBMaxN = 1024;       // largest n of the batched path
constexpr int kBMaxM = kBMaxBlocks * kNodeRows;

struct BProb {
    int m, n, lda, ldr;
    const float* A;
    const double* b;
    double* x;
    float* Rout;
    float* W; __half* Wh; int ldw;   // FP32 work matrix and its low-precision copy (rows padded)
    float* R; float* M; float* Mt; float* tmp;   // n x n, ld n
    __half* R12l; int ldr12;          // scaled low-precision R12 (columns padded to 16)
    int* eA; int* f;
    double* vec;                      // r, q (m each), t, p, s, u (n each)
    double* info;                     // 16 doubles
};

struct BArgs {
    BProb* probs;
    const int* order;
    int count;
    unsigned* queue;
    int target, max_iter, lowp;
    double tol;
    int* err;
};

struct BSmem {
    float red[kRedFloats];
    float Rs[32 * 33];
    float Rstk[kBMaxBlocks * 16 * 16];
    float Qt[kBMaxBlocks * 16 * 16];
    __align__(32) float wm[kPanelWarps][16 * 16];
    __align__(32) __half hs[kPanelWarps][16 * 16];
    float2 vs[kBMaxM];                // double-float staging of one vector
    double dred[kPanelWarps];
    float As[16][68];
    float Bs[16][68];
    int next;
};

__device__ __forceinline__ int round16(int v) { return (v + 15) & ~15; }

// The low-precision buffers are typed __half but hold TL (FP16 or BF16) bit patterns.
template <typename TL>
__device__ __forceinline__ void store_lp(__half* base, size_t idx, float v) {
    reinterpret_cast<TL*>(base)[idx] = LowPrec<TL>::from_float(v);
}

// ---- small CTA-wide helpers ------------------------------------------------------------
__device__ __forceinline__ double cta_sum(double v, BSmem& sm) {
    v = warp_sum_d(v);
    __syncthreads();
    if ((threadIdx.x & 31) == 0) sm.dred[threadIdx.x >> 5] = v;
    __syncthreads();
    double t = 0.0;
#pragma unroll
    for (int w = 0; w < kPanelWarps; ++w) t += sm.dred[w];
    __syncthreads();
    return t;
}

__device__ __forceinline__ void stage(const double* v, int len, BSmem& sm) {
    __syncthreads();
    for (int i = threadIdx.x; i < len; i += kPanelThreads) {
        float hi, lo;
        split_df(v[i], hi, lo);
        sm.vs[i] = make_float2(hi, lo);
    }
    __syncthreads();
}

// ---- panel (Eq. caqr) on one CTA --------------------------------------------------------
template <typename TL>
__device__ void panel_cta(const BProb& P, int c0, int w, BSmem& sm) {
    const int t = threadIdx.x, m = P.m;
    const int nb = (m + kNodeRows - 1) / kNodeRows;
    float v[kRPT][kBPw];
    for (int blk = 0; blk < nb; ++blk) {
        const int s = blk * (m / nb) + min(blk, m % nb);
        const int rows = m / nb + (blk < m % nb ? 1 : 0);
        for (int i = t; i < 32 * 33; i += kPanelThreads) sm.Rs[i] = 0.f;
#pragma unroll
        for (int r = 0; r < kRPT; ++r) {
            const int lr = t + r * kPanelThreads;
#pragma unroll
            for (int j = 0; j < kBPw; ++j)
                v[r][j] = (lr < rows && j < w && LLS_INB(s + lr < m && c0 + j < P.n))
                              ? P.W[(size_t)(s + lr) + (size_t)(c0 + j) * P.ldw] : 0.f;
        }
        __syncthreads();
        cgs2_block<kBPw>(v, w, sm.red, sm.Rs);
        const int off = kBPw - w;
#pragma unroll
        for (int r = 0; r < kRPT; ++r) {
            const int lr = t + r * kPanelThreads;
            if (lr >= rows) continue;
#pragma unroll
            for (int p = 0; p < kBPw; ++p) {
                const int j = p - off;
                if (j < 0 || !LLS_INB(s + lr < m && c0 + j < P.n)) continue;
                const size_t idx = (size_t)(s + lr) + (size_t)(c0 + j) * P.ldw;
                P.W[idx] = v[r][p];
                if (nb == 1) store_lp<TL>(P.Wh, idx, v[r][p]);
            }
        }
        if (nb == 1) {
            for (int i = t; i < w * w; i += kPanelThreads) {
                const int rr = i % w, cc = i / w;
                P.R[(size_t)(c0 + rr) + (size_t)(c0 + cc) * P.n] = rr <= cc ? sm.Rs[rr * 33 + cc] : 0.f;
            }
            __syncthreads();
            return;
        }
        for (int i = t; i < 256; i += kPanelThreads) {
            const int rr = i / 16, cc = i % 16;
            sm.Rstk[blk * 256 + i] = (rr < w && cc < w) ? sm.Rs[rr * 33 + cc] : 0.f;
        }
        __syncthreads();
    }
    // stack of nb R factors (nb * w rows) -> one more CGS2
    for (int i = t; i < 32 * 33; i += kPanelThreads) sm.Rs[i] = 0.f;
#pragma unroll
    for (int r = 0; r < kRPT; ++r) {
        const int rho = t + r * kPanelThreads;
        const int child = rho / w, rr = rho % w;
#pragma unroll
        for (int j = 0; j < kBPw; ++j)
            v[r][j] = (child < nb && j < w) ? sm.Rstk[child * 256 + rr * 16 + j] : 0.f;
    }
    __syncthreads();
    cgs2_block<kBPw>(v, w, sm.red, sm.Rs);
    const int off = kBPw - w;
#pragma unroll
    for (int r = 0; r < kRPT; ++r) {
        const int rho = t + r * kPanelThreads;
        if (rho < nb * w)
#pragma unroll
            for (int p = 0; p < kBPw; ++p)
                if (p >= off) sm.Qt[rho * 16 + (p - off)] = v[r][p];
    }
    for (int i = t; i < w * w; i += kPanelThreads) {
        const int rr = i % w, cc = i / w;
        P.R[(size_t)(c0 + rr) + (size_t)(c0 + cc) * P.n] = rr <= cc ? sm.Rs[rr * 33 + cc] : 0.f;
    }
    __syncthreads();
    // Q_block <- Q_block * (slice of the stack's Q)
    for (int blk = 0; blk < nb; ++blk) {
        const int s = blk * (m / nb) + min(blk, m % nb);
        const int rows = m / nb + (blk < m % nb ? 1 : 0);
        const float* T = sm.Qt + blk * w * 16;
        for (int lr = t; lr < rows; lr += kPanelThreads) {
            float q[kBPw];
#pragma unroll
            for (int k = 0; k < kBPw; ++k) q[k] = k < w ? P.W[(size_t)(s + lr) + (size_t)(c0 + k) * P.ldw] : 0.f;
            for (int j = 0; j < w; ++j) {
                float acc = 0.f;
#pragma unroll
                for (int k = 0; k < kBPw; ++k)
                    if (k < w) acc = fmaf(q[k], T[k * 16 + j], acc);
                const size_t idx = (size_t)(s + lr) + (size_t)(c0 + j) * P.ldw;
                P.W[idx] = acc;
                store_lp<TL>(P.Wh, idx, acc);
            }
        }
    }
    __syncthreads();
}

// ---- scale / cast of w columns of W into Wh (one warp per column) ------------------------
template <typename TL>
__device__ void cast_cols(const BProb& P, int c0, int w, int* exps, int lowp) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    for (int j = warp; j < w; j += kPanelWarps) {
        const float* col = P.W + (size_t)(c0 + j) * P.ldw;
        float mx = 0.f;
        for (int i = lane; i < P.m; i += 32) mx = fmaxf(mx, fabsf(col[i]));
        mx = warp_max_f(mx);
        const int e = lowp == 0 ? fp16_scale_exponent(mx) : 0;
        if (lane == 0) exps[j] = e;
        const float sc = pow2f(e);
        __half* out = P.Wh + (size_t)(c0 + j) * P.ldw;
        for (int i = lane; i < P.m; i += 32) store_lp<TL>(out, i, col[i] * sc);
    }
    __syncthreads();
}

// ---- the two products of a recursion step (tensor cores, warp-level fragments) ----------
// TL is __half or __nv_bfloat16; the buffers are declared __half and reinterpreted.
template <typename TL>
__device__ void proj_and_update(const BProb& P, int c0, int w1, int w2, int lowp, BSmem& sm) {
    typedef typename std::conditional<std::is_same<TL, __half>::value, half, __nv_bfloat16>::type FT;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int m16 = round16(P.m);
    const FT* Wh = reinterpret_cast<const FT*>(P.Wh);
    // R12 = Q1l^T A2l (w1 x w2), unscaled by 2^-e_j, into R; K = m (rows >= m are zero)
    const int ti_n = w1 / 16, tj_n = (w2 + 15) / 16;
    for (int tt = warp; tt < ti_n * tj_n; tt += kPanelWarps) {
        const int ti = tt % ti_n, tj = tt / ti_n;
        const bool ragged = 16 * tj + 16 > w2;
        wmma::fragment<wmma::accumulator, 16, 16, 16, float> acc;
        wmma::fill_fragment(acc, 0.f);
        for (int k0 = 0; k0 < m16; k0 += 16) {
            wmma::fragment<wmma::matrix_a, 16, 16, 16, FT, wmma::row_major> fa;
            wmma::fragment<wmma::matrix_b, 16, 16, 16, FT, wmma::col_major> fb;
            wmma::load_matrix_sync(fa, Wh + (size_t)(c0 + 16 * ti) * P.ldw + k0, P.ldw);
            if (!ragged) {
                wmma::load_matrix_sync(fb, Wh + (size_t)(c0 + w1 + 16 * tj) * P.ldw + k0, P.ldw);
            } else {
                FT* hs = reinterpret_cast<FT*>(sm.hs[warp]);
                for (int e = lane; e < 256; e += 32) {
                    const int kk = e % 16, cc = e / 16;
                    hs[e] = (16 * tj + cc < w2) ? Wh[(size_t)(c0 + w1 + 16 * tj + cc) * P.ldw + k0 + kk]
                                                : LowPrec<TL>::from_float(0.f);
                }
                __syncwarp();
                wmma::load_matrix_sync(fb, hs, 16);
                __syncwarp();
            }
            wmma::mma_sync(acc, fa, fb, acc);
        }
        wmma::store_matrix_sync(sm.wm[warp], acc, 16, wmma::mem_col_major);
        __syncwarp();
        for (int e = lane; e < 256; e += 32) {
            const int rr = e % 16, cc = e / 16;
            const int j = 16 * tj + cc;
            if (j < w2)
                P.R[(size_t)(c0 + 16 * ti + rr) + (size_t)(c0 + w1 + j) * P.n] = sm.wm[warp][e] * pow2f(-P.eA[j]);
        }
        __syncwarp();
    }
    __syncthreads();
    // R12l = round(R12 * 2^f_j), f_j from the column maximum (one warp per column)
    FT* R12l = reinterpret_cast<FT*>(P.R12l);
    const int w2p = round16(w2);
    for (int j = warp; j < w2p; j += kPanelWarps) {
        if (j >= w2) {
            for (int i = lane; i < w1; i += 32) R12l[i + (size_t)j * P.ldr12] = LowPrec<TL>::from_float(0.f);
            continue;
        }
        const float* col = P.R + (size_t)c0 + (size_t)(c0 + w1 + j) * P.n;
        float mx = 0.f;
        for (int i = lane; i < w1; i += 32) mx = fmaxf(mx, fabsf(col[i]));
        mx = warp_max_f(mx);
        const int fe = lowp == 0 ? fp16_scale_exponent(mx) : 0;
        if (lane == 0) P.f[j] = fe;
        const float sc = pow2f(fe);
        for (int i = lane; i < w1; i += 32) R12l[i + (size_t)j * P.ldr12] = LowPrec<TL>::from_float(col[i] * sc);
    }
    __syncthreads();
    // A2 -= (Q1l R12l) 2^-f_j, tiles of 16 rows x 16 columns
    const int mi_n = m16 / 16;
    for (int tt = warp; tt < mi_n * tj_n; tt += kPanelWarps) {
        const int ti = tt % mi_n, tj = tt / mi_n;
        wmma::fragment<wmma::accumulator, 16, 16, 16, float> acc;
        wmma::fill_fragment(acc, 0.f);
        for (int k0 = 0; k0 < w1; k0 += 16) {
            wmma::fragment<wmma::matrix_a, 16, 16, 16, FT, wmma::col_major> fa;
            wmma::fragment<wmma::matrix_b, 16, 16, 16, FT, wmma::col_major> fb;
            wmma::load_matrix_sync(fa, Wh + (size_t)(c0 + k0) * P.ldw + 16 * ti, P.ldw);
            wmma::load_matrix_sync(fb, R12l + (size_t)(16 * tj) * P.ldr12 + k0, P.ldr12);
            wmma::mma_sync(acc, fa, fb, acc);
        }
        wmma::store_matrix_sync(sm.wm[warp], acc, 16, wmma::mem_col_major);
        __syncwarp();
        for (int e = lane; e < 256; e += 32) {
            const int rr = e % 16, cc = e / 16;
            const int i = 16 * ti + rr, j = 16 * tj + cc;
            if (i < P.m && j < w2) {
                const size_t idx = (size_t)i + (size_t)(c0 + w1 + j) * P.ldw;
                P.W[idx] = P.W[idx] - sm.wm[warp][e] * pow2f(-P.f[j]);
            }
        }
        __syncwarp();
    }
    __syncthreads();
}

__device__ __forceinline__ int split_point_dev(int w) { return kBPw * ((w + 2 * kBPw - 1) / (2 * kBPw)); }

// Alg. 2, depth first, with an explicit stack (every thread runs the same control flow).
template <typename TL>
__device__ void rgsqrf_cta(const BProb& P, int lowp, BSmem& sm) {
    struct Frame { int c0, w, stage; };
    Frame st[16];
    int sp = 0;
    st[0] = {0, P.n, 0};
    while (sp >= 0) {
        Frame& fr = st[sp];
        if (fr.w <= kBPw) {
            panel_cta<TL>(P, fr.c0, fr.w, sm);
            --sp;
            continue;
        }
        const int w1 = split_point_dev(fr.w), w2 = fr.w - w1;
        if (fr.stage == 0) {
            fr.stage = 1;
            st[++sp] = {fr.c0, w1, 0};
        } else if (fr.stage == 1) {
            fr.stage = 2;
            cast_cols<TL>(P, fr.c0 + w1, w2, P.eA, lowp);
            proj_and_update<TL>(P, fr.c0, w1, w2, lowp, sm);
            st[++sp] = {fr.c0 + w1, w2, 0};
        } else {
            --sp;
        }
    }
}

// ---- R^{-1} on one CTA (Eq. recqr block inverse) ----------------------------------------
// C = alpha * A B (M x N, K), FP32 tiles of 64 x 64 in shared memory.
__device__ void cta_gemm(int Mr, int Nc, int K, float alpha, const float* A, int lda, const float* B, int ldb,
                         float* C, int ldc, BSmem& sm) {
    const int t = threadIdx.x;
    const int ti = (t % 16) * 4, tj = (t / 16) * 4;
    for (int i0 = 0; i0 < Mr; i0 += 64)
        for (int j0 = 0; j0 < Nc; j0 += 64) {
            float acc[4][4] = {};
            for (int k0 = 0; k0 < K; k0 += 16) {
                __syncthreads();
#pragma unroll
                for (int r = 0; r < 4; ++r) {
                    const int idx = t + r * 256;
                    const int ii = idx % 64, kk = idx / 64;
                    sm.As[kk][ii] = (i0 + ii < Mr && k0 + kk < K) ? A[(size_t)(i0 + ii) + (size_t)(k0 + kk) * lda] : 0.f;
                    const int kk2 = idx % 16, jj = idx / 16;
                    sm.Bs[kk2][jj] = (j0 + jj < Nc && k0 + kk2 < K) ? B[(size_t)(k0 + kk2) + (size_t)(j0 + jj) * ldb] : 0.f;
                }
                __syncthreads();
#pragma unroll
                for (int kk = 0; kk < 16; ++kk) {
                    float av[4], bv[4];
#pragma unroll
                    for (int u = 0; u < 4; ++u) { av[u] = sm.As[kk][ti + u]; bv[u] = sm.Bs[kk][tj + u]; }
#pragma unroll
                    for (int u = 0; u < 4; ++u)
#pragma unroll
                        for (int vv = 0; vv < 4; ++vv) acc[u][vv] = fmaf(av[u], bv[vv], acc[u][vv]);
                }
            }
#pragma unroll
            for (int vv = 0; vv < 4; ++vv)
#pragma unroll
                for (int u = 0; u < 4; ++u) {
                    const int i = i0 + ti + u, j = j0 + tj + vv;
                    if (i < Mr && j < Nc) C[(size_t)i + (size_t)j * ldc] = alpha * acc[u][vv];
                }
        }
    __syncthreads();
}

__device__ void trinv_cta(const BProb& P, BSmem& sm, int* err) {
    const int n = P.n, lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    for (size_t e = threadIdx.x; e < (size_t)n * n; e += kPanelThreads) P.M[e] = 0.f;
    __syncthreads();
    // leaves: columns [16 k, 16 k + w); one warp per leaf, one lane per column of the inverse
    const int nleaf = (n + kBPw - 1) / kBPw;
    for (int lf = warp; lf < nleaf; lf += kPanelWarps) {
        // leaves of the split tree are the 16-column blocks (split points are multiples of 16)
        const int c0 = lf * kBPw, w = min(kBPw, n - c0);
        const int j = lane;
        if (j < w) {
            float mcol[kBPw];
            for (int i = w - 1; i >= 0; --i) {
                float s = (i == j) ? 1.f : 0.f;
                for (int k = i + 1; k <= j; ++k) s = fmaf(-P.R[(size_t)(c0 + i) + (size_t)(c0 + k) * n], mcol[k], s);
                const float d = P.R[(size_t)(c0 + i) + (size_t)(c0 + i) * n];
                if (!(d != 0.f) || !isfinite(d)) atomicCAS(err, DEV_OK, DEV_SINGULAR);
                mcol[i] = i <= j ? s / d : 0.f;
            }
            for (int i = 0; i <= j; ++i) P.M[(size_t)(c0 + i) + (size_t)(c0 + j) * n] = mcol[i];
        }
    }
    __syncthreads();
    // internal nodes in post-order: M12 = -M11 (R12 M22)
    struct Frame { int c0, w, stage; };
    Frame st[16];
    int sp = 0;
    st[0] = {0, n, 0};
    while (sp >= 0) {
        Frame& fr = st[sp];
        if (fr.w <= kBPw) { --sp; continue; }
        const int w1 = split_point_dev(fr.w), w2 = fr.w - w1;
        if (fr.stage == 0) { fr.stage = 1; st[++sp] = {fr.c0, w1, 0}; continue; }
        if (fr.stage == 1) { fr.stage = 2; st[++sp] = {fr.c0 + w1, w2, 0}; continue; }
        const int c0 = fr.c0;
        cta_gemm(w1, w2, w2, 1.f, P.R + (size_t)c0 + (size_t)(c0 + w1) * n, n,
                 P.M + (size_t)(c0 + w1) + (size_t)(c0 + w1) * n, n, P.tmp, w1, sm);
        cta_gemm(w1, w2, w1, -1.f, P.M + (size_t)c0 + (size_t)c0 * n, n, P.tmp, w1,
                 P.M + (size_t)c0 + (size_t)(c0 + w1) * n, n, sm);
        --sp;
    }
    for (size_t e = threadIdx.x; e < (size_t)n * n; e += kPanelThreads) {
        const int i = (int)(e % n), j = (int)(e / n);
        P.Mt[(size_t)j + (size_t)i * n] = P.M[e];
    }
    __syncthreads();
}

// ---- CGLS (Alg. 5) on one CTA ----------------------------------------------------------
// out_c = sum over rows [lo, hi) of column c of X (n x n) times the staged vector
__device__ double cta_tri_gemv(const float* X, int n, bool upper, double* out, BSmem& sm) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    double sq = 0.0;
    for (int c = warp; c < n; c += kPanelWarps) {
        const int lo = upper ? 0 : c, hi = upper ? c + 1 : n;
        float s = 0.f, cc = 0.f;
        for (int r = lo + lane; r < hi; r += 32) {
            const float2 v = sm.vs[r];
            dot2_step(s, cc, X[(size_t)r + (size_t)c * n], v.x, v.y);
        }
        warp_sum_df(s, cc);
        if (lane == 0) { const double v = join_df(s, cc); out[c] = v; sq += v * v; }
    }
    return sq;
}

// out = A v (v staged in sm.vs), or b - A v when bvec is given; returns the thread's part of
// ||out||^2. Threads own rows (coalesced column reads), four rows at a time.
__device__ double cta_a_times(const BProb& P, double* out, const double* bvec, BSmem& sm) {
    double sq = 0.0;
    for (int i0 = 0; i0 < P.m; i0 += 4 * kPanelThreads) {
        float s[4] = {0.f, 0.f, 0.f, 0.f}, c[4] = {0.f, 0.f, 0.f, 0.f};
        for (int j = 0; j < P.n; ++j) {
            const float2 v = sm.vs[j];
            const float* col = P.A + (size_t)j * P.lda;
#pragma unroll
            for (int r = 0; r < 4; ++r) {
                const int i = i0 + threadIdx.x + r * kPanelThreads;
                if (i < P.m) dot2_step(s[r], c[r], col[i], v.x, v.y);
            }
        }
#pragma unroll
        for (int r = 0; r < 4; ++r) {
            const int i = i0 + threadIdx.x + r * kPanelThreads;
            if (i < P.m) {
                double val = join_df(s[r], c[r]);
                if (bvec) val = bvec[i] - val;
                out[i] = val;
                sq += val * val;
            }
        }
    }
    return sq;
}

// out = A^T v (v of length m staged in sm.vs): one warp per column; returns ||out||^2 part.
__device__ double cta_at_times(const BProb& P, double* out, BSmem& sm) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    double sq = 0.0;
    for (int j = warp; j < P.n; j += kPanelWarps) {
        const float* col = P.A + (size_t)j * P.lda;
        float s = 0.f, c = 0.f;
        for (int i = lane; i < P.m; i += 32) {
            const float2 v = sm.vs[i];
            dot2_step(s, c, col[i], v.x, v.y);
        }
        warp_sum_df(s, c);
        if (lane == 0) { const double v = join_df(s, c); out[j] = v; sq += v * v; }
    }
    return sq;
}

__device__ double cta_fro2(const float* X, int rows, int cols, int ld, BSmem& sm) {
    float s = 0.f, c = 0.f;
    for (size_t e = threadIdx.x; e < (size_t)rows * cols; e += kPanelThreads) {
        const float v = X[(e % rows) + (e / rows) * (size_t)ld];
        dot2_step(s, c, v, v, 0.f);
    }
    return cta_sum(join_df(s, c), sm);
}

__device__ void cgls_cta(const BProb& P, const BArgs& g, BSmem& sm) {
    const int m = P.m, n = P.n;
    double* r = P.vec;
    double* q = r + m;
    double* t = q + m;
    double* p = t + n;
    double* s = p + n;
    double* u = s + n;
    double* x = P.x;
    const double anorm = sqrt(cta_fro2(P.A, m, n, P.lda, sm));
    const double mnorm = sqrt(cta_fro2(P.M, n, n, n, sm));
    for (int i = threadIdx.x; i < m; i += kPanelThreads) r[i] = P.b[i];
    for (int j = threadIdx.x; j < n; j += kPanelThreads) x[j] = 0.0;
    int iters = 0, status = 1, passes = 0;
    double eta = 0.0, fwd = 0.0, rn2 = 0.0, un2 = 0.0, xn2 = 0.0;
    for (int restart = 0; restart <= 2; ++restart) {
        if (restart > 0) {     // fresh residual r = b - A x
            stage(x, n, sm);
            rn2 = cta_sum(cta_a_times(P, r, P.b, sm), sm);
            ++passes;
        } else {
            double v = 0.0;
            for (int i = threadIdx.x; i < m; i += kPanelThreads) v += P.b[i] * P.b[i];
            rn2 = cta_sum(v, sm);
        }
        stage(r, m, sm);
        un2 = cta_sum(cta_at_times(P, u, sm), sm);
        ++passes;
        stage(u, n, sm);
        double gamma = cta_sum(cta_tri_gemv(P.M, n, true, s, sm), sm);
        double xs = 0.0;
        for (int j = threadIdx.x; j < n; j += kPanelThreads) xs += x[j] * x[j];
        xn2 = cta_sum(xs, sm);
        const double xn = sqrt(xn2), sn = sqrt(gamma);
        eta = xn > 0.0 ? sn / (anorm * xn) : (sn == 0.0 ? 0.0 : INFINITY);
        fwd = xn > 0.0 ? mnorm * sn / xn : (sn == 0.0 ? 0.0 : INFINITY);
        if ((g.target == LLS_TARGET_FP64 ? eta : fwd) <= g.tol) { status = 0; break; }
        if (iters >= g.max_iter || restart == 2) break;
        for (int j = threadIdx.x; j < n; j += kPanelThreads) p[j] = s[j];
        while (iters < g.max_iter) {
            stage(p, n, sm);
            cta_tri_gemv(P.Mt, n, false, t, sm);
            stage(t, n, sm);
            const double delta = cta_sum(cta_a_times(P, q, nullptr, sm), sm);
            ++passes;
            ++iters;
            if (!(delta > 0.0)) break;
            const double alpha = gamma / delta;
            double xs2 = 0.0;
            for (int j = threadIdx.x; j < n; j += kPanelThreads) { x[j] += alpha * t[j]; xs2 += x[j] * x[j]; }
            for (int i = threadIdx.x; i < m; i += kPanelThreads) r[i] -= alpha * q[i];
            const double xnn = sqrt(cta_sum(xs2, sm));
            stage(r, m, sm);
            cta_at_times(P, u, sm);
            ++passes;
            stage(u, n, sm);
            const double gnew = cta_sum(cta_tri_gemv(P.M, n, true, s, sm), sm);
            const double beta = gnew / gamma;
            gamma = gnew;
            for (int j = threadIdx.x; j < n; j += kPanelThreads) p[j] = s[j] + beta * p[j];
            const double sn2 = sqrt(gnew);
            const double e1 = xnn > 0.0 ? sn2 / (anorm * xnn) : INFINITY;
            const double f1 = xnn > 0.0 ? mnorm * sn2 / xnn : INFINITY;
            if ((g.target == LLS_TARGET_FP64 ? e1 : f1) <= g.tol) break;
        }
    }
    if (threadIdx.x == 0) {
        P.info[0] = iters; P.info[1] = eta; P.info[2] = fwd; P.info[3] = sqrt(rn2);
        P.info[4] = sqrt(un2); P.info[5] = anorm; P.info[6] = sqrt(xn2); P.info[7] = status;
        P.info[10] = passes; P.info[11] = 0;
    }
    __syncthreads();
}

// ---- the persistent kernel ------------------------------------------------------------
template <typename TL>
__global__ void __launch_bounds__(kPanelThreads, 1)
batched_lls_kernel(BArgs g) {
    extern __shared__ __align__(16) unsigned char b_smem_raw[];
    BSmem& sm = *reinterpret_cast<BSmem*>(b_smem_raw);
    for (;;) {
        if (threadIdx.x == 0) sm.next = (int)atomicAdd(g.queue, 1u);
        __syncthreads();
        const int k = sm.next;
        __syncthreads();
        if (k >= g.count) return;
        if (!LLS_INB(g.order[k] >= 0 && g.order[k] < g.count)) continue;
        const BProb P = g.probs[g.order[k]];
        // W = A, low-precision rows m..ldw-1 zero (the tensor-core tiles read whole 16-row blocks)
        for (size_t e = threadIdx.x; e < (size_t)P.ldw * P.n; e += kPanelThreads) {
            const int i = (int)(e % P.ldw), j = (int)(e / P.ldw);
            P.W[e] = i < P.m ? P.A[(size_t)i + (size_t)j * P.lda] : 0.f;
            if (i >= P.m) P.Wh[e] = __float2half(0.f);
        }
        __syncthreads();
        rgsqrf_cta<TL>(P, g.lowp, sm);
        if (P.Rout)   // only the upper triangle of the work copy of R is ever written
            for (size_t e = threadIdx.x; e < (size_t)P.n * P.n; e += kPanelThreads) {
                const int i = (int)(e % P.n), j = (int)(e / P.n);
                P.Rout[(size_t)i + (size_t)j * P.ldr] = i <= j ? P.R[e] : 0.f;
            }
        __syncthreads();
        int* perr = reinterpret_cast<int*>(P.info + 12);
        if (threadIdx.x == 0) *perr = 0;
        __syncthreads();
        trinv_cta(P, sm, perr);
        if (*(volatile int*)perr != 0) {
            if (threadIdx.x == 0) { P.info[7] = -2; P.info[0] = 0; }
            __syncthreads();
            continue;
        }
        cgls_cta(P, g, sm);
    }
}

// ---- the adjoint of a batch of solves, one persistent launch ------------------------------
// Each CTA takes whole problems from the work queue and runs, for its problem, the textbook
// sensitivity of x* = (A^T A)^{-1} A^T b (the paper has none): M = R^{-1} from the solve's R
// (the block inverse above), z = (A^T A)^{-1} g by CG preconditioned with M M^T,
//   res = g, u = M^T res, y = M u, rho = ||u||^2, p = y
//   loop: q = A p, w = A^T q, alpha = rho / (p . w), z += alpha p, res -= alpha w,
//         u = M^T res, rho' = ||u||^2, beta = rho' / rho, y = M u, p = y + beta p
//   until ||M^T res|| <= tol ||M^T g||,
// then r = b - A x, dL/db = A z and dL/dA = r z^T - (A z) x^T written in one sweep. The
// products with A and M use the same compensated (double-float) dot products as the solve.
struct AProb {
    int m, n, lda, ldr, ldga;
    const float* A; const double* b; const double* x; const double* g; const float* Rin;
    float* gA; double* gb;
    float* R; float* M; float* Mt; float* tmp;   // n x n, ld n (R: the copy of Rin)
    double* vec;                                 // res, u, y, p, w, z (n each); q, r, az (m each)
    double* info;                                // 16 doubles: iterations, status, ...
};

struct AArgs {
    AProb* probs;
    const int* order;
    int count;
    unsigned* queue;
    double tol;
    int max_iter;
};

__device__ void adjoint_cta(const AProb& Q, const AArgs& g, BSmem& sm) {
    const int m = Q.m, n = Q.n;
    // the building blocks above take their sizes and pointers from a BProb
    BProb P;
    P.m = m; P.n = n; P.lda = Q.lda; P.A = Q.A; P.R = Q.R; P.M = Q.M; P.Mt = Q.Mt; P.tmp = Q.tmp;
    double* res = Q.vec;
    double* u = res + n;
    double* y = u + n;
    double* p = y + n;
    double* w = p + n;
    double* z = w + n;
    double* q = z + n;
    double* r = q + m;
    double* az = r + m;
    for (size_t e = threadIdx.x; e < (size_t)n * n; e += kPanelThreads) {
        const int i = (int)(e % n), j = (int)(e / n);
        Q.R[e] = i <= j ? Q.Rin[(size_t)i + (size_t)j * Q.ldr] : 0.f;
    }
    __syncthreads();
    int* perr = reinterpret_cast<int*>(Q.info + 12);
    if (threadIdx.x == 0) *perr = 0;
    __syncthreads();
    trinv_cta(P, sm, perr);
    if (*(volatile int*)perr != 0) {
        if (threadIdx.x == 0) { Q.info[0] = 0; Q.info[7] = -2; }
        __syncthreads();
        return;
    }
    for (int j = threadIdx.x; j < n; j += kPanelThreads) { res[j] = Q.g[j]; z[j] = 0.0; }
    stage(res, n, sm);
    double rho = cta_sum(cta_tri_gemv(Q.M, n, true, u, sm), sm);
    const double rho0 = rho;
    stage(u, n, sm);
    cta_tri_gemv(Q.Mt, n, false, y, sm);
    __syncthreads();
    for (int j = threadIdx.x; j < n; j += kPanelThreads) p[j] = y[j];
    int iters = 0, status = rho0 > 0.0 ? 1 : 0;
    while (status != 0 && iters < g.max_iter) {
        stage(p, n, sm);
        cta_a_times(P, q, nullptr, sm);                 // q = A p
        stage(q, m, sm);
        cta_at_times(P, w, sm);                         // w = A^T q
        __syncthreads();
        double pw = 0.0;
        for (int j = threadIdx.x; j < n; j += kPanelThreads) pw += p[j] * w[j];
        pw = cta_sum(pw, sm);
        ++iters;
        if (!(pw > 0.0)) { status = 0; break; }
        const double alpha = rho / pw;
        for (int j = threadIdx.x; j < n; j += kPanelThreads) { z[j] += alpha * p[j]; res[j] -= alpha * w[j]; }
        stage(res, n, sm);
        const double rnew = cta_sum(cta_tri_gemv(Q.M, n, true, u, sm), sm);
        const double beta = rnew / rho;
        rho = rnew;
        stage(u, n, sm);
        cta_tri_gemv(Q.Mt, n, false, y, sm);
        __syncthreads();
        for (int j = threadIdx.x; j < n; j += kPanelThreads) p[j] = y[j] + beta * p[j];
        if (sqrt(rho) <= g.tol * sqrt(rho0)) status = 0;
    }
    // r = b - A x, A z
    stage(Q.x, n, sm);
    cta_a_times(P, r, Q.b, sm);
    stage(z, n, sm);
    cta_a_times(P, az, nullptr, sm);
    __syncthreads();
    for (int i = threadIdx.x; i < m; i += kPanelThreads) Q.gb[i] = az[i];
    // dL/dA = r z^T - (A z) x^T, column by column (coalesced over rows)
    for (int j = 0; j < n; ++j) {
        const double zj = z[j], xj = Q.x[j];
        float* col = Q.gA + (size_t)j * Q.ldga;
        for (int i = threadIdx.x; i < m; i += kPanelThreads) col[i] = (float)(r[i] * zj - az[i] * xj);
    }
    if (threadIdx.x == 0) { Q.info[0] = iters; Q.info[7] = status; }
    __syncthreads();
}

__global__ void __launch_bounds__(kPanelThreads, 1)
batched_adjoint_kernel(AArgs g) {
    extern __shared__ __align__(16) unsigned char b_smem_raw[];
    BSmem& sm = *reinterpret_cast<BSmem*>(b_smem_raw);
    for (;;) {
        if (threadIdx.x == 0) sm.next = (int)atomicAdd(g.queue, 1u);
        __syncthreads();
        const int k = sm.next;
        __syncthreads();
        if (k >= g.count) return;
        if (!LLS_INB(g.order[k] >= 0 && g.order[k] < g.count)) continue;
        const AProb Q = g.probs[g.order[k]];
        adjoint_cta(Q, g, sm);
    }
}

// ---------------------------------------------------------------------------------------
// Host side
// ---------------------------------------------------------------------------------------
struct BLayout {
    size_t table, order, queue, info, total;
    std::vector<size_t> off;   // per-problem base offset
};

static size_t prob_bytes(int m, int n) {
    const size_t ldw = align_up((size_t)m, 64);
    const size_t n2 = (size_t)n * n;
    const size_t r12 = align_up((size_t)(n / 2 + kBPw), 16);
    size_t b = 0;
    b += align_up(ldw * n * 4, 256);          // W
    b += align_up(ldw * n * 2, 256);          // Wh
    b += 4 * align_up(n2 * 4, 256);           // R, M, Mt, tmp
    b += align_up(r12 * r12 * 2, 256);        // R12l
    b += 2 * align_up((size_t)n * 4, 256);    // eA, f
    b += align_up(((size_t)2 * m + 4 * n) * 8, 256);   // vectors
    return b;
}

static void b_layout(int batch, const int* m, const int* n, BLayout& L) {
    size_t o = 0;
    L.table = o; o = align_up(o + sizeof(BProb) * batch, 256);
    L.order = o; o = align_up(o + sizeof(int) * batch, 256);
    L.queue = o; o = align_up(o + 256, 256);
    L.info = o; o = align_up(o + sizeof(double) * 16 * batch, 256);
    L.off.resize(batch);
    for (int i = 0; i < batch; ++i) { L.off[i] = o; o += prob_bytes(m[i], n[i]); }
    L.total = o;
}

bool batched_supported(int m, int n) { return n >= 1 && m >= n && m <= kBMaxM && n <= kBMaxN; }

size_t batched_workspace_bytes(int batch, const int* m, const int* n) {
    BLayout L;
    b_layout(batch, m, n, L);
    return L.total;
}

double* batched_info_ptr(void* ws, int batch, const int* m, const int* n) {
    BLayout L;
    b_layout(batch, m, n, L);
    return (double*)((char*)ws + L.info);
}

// Fill and upload the problem table (host -> workspace; ordinary stream-ordered copies).
int batched_upload(int batch, const int* m, const int* n, const float* const* A, const int* lda,
                   const double* const* b, double* const* x, float* const* Rout, const int* ldr,
                   void* ws, size_t ws_bytes, cudaStream_t st) {
    BLayout L;
    b_layout(batch, m, n, L);
    if (L.total > ws_bytes) return LLS_ERR_WORKSPACE;
    char* base = (char*)ws;
    std::vector<BProb> table(batch);
    std::vector<int> order(batch);
    for (int i = 0; i < batch; ++i) {
        BProb& P = table[i];
        const size_t ldw = align_up((size_t)m[i], 64);
        const size_t n2 = (size_t)n[i] * n[i];
        char* q = base + L.off[i];
        auto take = [&](size_t bytes) { char* r = q; q += align_up(bytes, 256); return r; };
        P.m = m[i]; P.n = n[i]; P.lda = lda[i];
        P.Rout = Rout ? Rout[i] : nullptr;
        P.ldr = P.Rout ? ldr[i] : n[i];
        P.A = A[i]; P.b = b[i]; P.x = x[i];
        P.ldw = (int)ldw;
        P.W = (float*)take(ldw * n[i] * 4);
        P.Wh = (__half*)take(ldw * n[i] * 2);
        P.R = (float*)take(n2 * 4); P.M = (float*)take(n2 * 4); P.Mt = (float*)take(n2 * 4); P.tmp = (float*)take(n2 * 4);
        const size_t r12d = align_up((size_t)(n[i] / 2 + kBPw), 16);
        P.ldr12 = (int)r12d;
        P.R12l = (__half*)take(r12d * r12d * 2);
        P.eA = (int*)take((size_t)n[i] * 4); P.f = (int*)take((size_t)n[i] * 4);
        P.vec = (double*)take(((size_t)2 * m[i] + 4 * n[i]) * 8);
        P.info = (double*)(base + L.info) + (size_t)16 * i;
        order[i] = i;
    }
    // largest estimated cost first (QR ~ m n^2, Krylov ~ m n per iteration)
    std::stable_sort(order.begin(), order.end(), [&](int a, int c) {
        return (double)m[a] * n[a] * (n[a] + 64.0) > (double)m[c] * n[c] * (n[c] + 64.0);
    });
    LLS_CUDA_TRY(cudaMemcpyAsync(base + L.table, table.data(), sizeof(BProb) * batch, cudaMemcpyHostToDevice, st));
    LLS_CUDA_TRY(cudaMemcpyAsync(base + L.order, order.data(), sizeof(int) * batch, cudaMemcpyHostToDevice, st));
    return LLS_OK;
}

// The persistent launch over an uploaded table (capturable in a CUDA graph).
int batched_execute(int batch, const int* m, const int* n, void* ws, const lls_options& o, int ctas_per_sm,
                    cudaStream_t st) {
    BLayout L;
    b_layout(batch, m, n, L);
    char* base = (char*)ws;
    LLS_CUDA_TRY(cudaMemsetAsync(base + L.queue, 0, 256, st));
    LLS_CUDA_TRY(cudaMemsetAsync(base + L.info, 0, sizeof(double) * 16 * batch, st));
    BArgs g;
    g.probs = (BProb*)(base + L.table);
    g.order = (const int*)(base + L.order);
    g.count = batch;
    g.queue = (unsigned*)(base + L.queue);
    g.target = o.target; g.max_iter = o.max_iter; g.tol = o.tol;
    g.lowp = o.gemm_prec == LLS_PREC_BF16 ? 1 : 0;
    g.err = nullptr;
    const size_t smem = sizeof(BSmem);
    int dev = 0, sms = 0, per = 0;
    LLS_CUDA_TRY(cudaGetDevice(&dev));
    LLS_CUDA_TRY(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    auto kern = g.lowp == 0 ? batched_lls_kernel<__half> : batched_lls_kernel<__nv_bfloat16>;
    LLS_CUDA_TRY(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    LLS_CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, kern, kPanelThreads, smem));
    if (per < 1) return LLS_ERR_UNSUPPORTED;
    if (ctas_per_sm > 0 && ctas_per_sm < per) per = ctas_per_sm;
    int grid = sms * per;
    if (grid > batch) grid = batch;
    kern<<<grid, kPanelThreads, smem, st>>>(g);
    LLS_LAUNCH_CHECK("batched_lls", st);
    return LLS_OK;
}

}  // namespace lls

// ---- the batched adjoint: workspace, upload and launch -----------------------------------
namespace lls {

static size_t adj_prob_bytes(int m, int n) {
    const size_t n2 = (size_t)n * n;
    return 4 * align_up(n2 * 4, 256) + align_up(((size_t)3 * m + 6 * n) * 8, 256) + 256;
}

struct ALayout {
    size_t table, order, queue, info, total;
    std::vector<size_t> off;
};

static void a_layout(int batch, const int* m, const int* n, ALayout& L) {
    size_t o = 0;
    L.table = o; o = align_up(o + sizeof(AProb) * batch, 256);
    L.order = o; o = align_up(o + sizeof(int) * batch, 256);
    L.queue = o; o = align_up(o + 256, 256);
    L.info = o; o = align_up(o + sizeof(double) * 16 * batch, 256);
    L.off.resize(batch);
    for (int i = 0; i < batch; ++i) { L.off[i] = o; o += adj_prob_bytes(m[i], n[i]); }
    L.total = o;
}

size_t batched_adjoint_workspace_bytes(int batch, const int* m, const int* n) {
    ALayout L;
    a_layout(batch, m, n, L);
    return L.total;
}

int batched_adjoint(int batch, const int* m, const int* n, const float* const* A, const int* lda,
                    const double* const* b, const double* const* x, const float* const* R, const int* ldr,
                    const double* const* grad_x, float* const* grad_A, const int* ldga, double* const* grad_b,
                    void* ws, size_t ws_bytes, double tol, int max_iter, cudaStream_t st) {
    ALayout L;
    a_layout(batch, m, n, L);
    if (L.total > ws_bytes) return LLS_ERR_WORKSPACE;
    char* base = (char*)ws;
    std::vector<AProb> table(batch);
    std::vector<int> order(batch);
    for (int i = 0; i < batch; ++i) {
        AProb& Q = table[i];
        const size_t n2 = (size_t)n[i] * n[i];
        char* q = base + L.off[i];
        auto take = [&](size_t bytes) { char* r = q; q += align_up(bytes, 256); return r; };
        Q.m = m[i]; Q.n = n[i]; Q.lda = lda[i]; Q.ldr = ldr[i]; Q.ldga = ldga[i];
        Q.A = A[i]; Q.b = b[i]; Q.x = x[i]; Q.g = grad_x[i]; Q.Rin = R[i];
        Q.gA = grad_A[i]; Q.gb = grad_b[i];
        Q.R = (float*)take(n2 * 4); Q.M = (float*)take(n2 * 4); Q.Mt = (float*)take(n2 * 4);
        Q.tmp = (float*)take(n2 * 4);
        Q.vec = (double*)take(((size_t)3 * m[i] + 6 * n[i]) * 8);
        Q.info = (double*)(base + L.info) + (size_t)16 * i;
        order[i] = i;
    }
    // largest first: CG costs about m n per iteration, the inverse about n^3 / 3
    std::stable_sort(order.begin(), order.end(), [&](int a, int c) {
        return (double)m[a] * n[a] * 40.0 + (double)n[a] * n[a] * n[a] > (double)m[c] * n[c] * 40.0 + (double)n[c] * n[c] * n[c];
    });
    LLS_CUDA_TRY(cudaMemcpyAsync(base + L.table, table.data(), sizeof(AProb) * batch, cudaMemcpyHostToDevice, st));
    LLS_CUDA_TRY(cudaMemcpyAsync(base + L.order, order.data(), sizeof(int) * batch, cudaMemcpyHostToDevice, st));
    LLS_CUDA_TRY(cudaMemsetAsync(base + L.queue, 0, 256, st));
    LLS_CUDA_TRY(cudaMemsetAsync(base + L.info, 0, sizeof(double) * 16 * batch, st));
    AArgs g;
    g.probs = (AProb*)(base + L.table);
    g.order = (const int*)(base + L.order);
    g.count = batch;
    g.queue = (unsigned*)(base + L.queue);
    g.tol = tol;
    g.max_iter = max_iter;
    const size_t smem = sizeof(BSmem);
    int dev = 0, sms = 0, per = 0;
    LLS_CUDA_TRY(cudaGetDevice(&dev));
    LLS_CUDA_TRY(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    LLS_CUDA_TRY(cudaFuncSetAttribute(batched_adjoint_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    LLS_CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, batched_adjoint_kernel, kPanelThreads, smem));
    if (per < 1) return LLS_ERR_UNSUPPORTED;
    int grid = sms * per;
    if (grid > batch) grid = batch;
    batched_adjoint_kernel<<<grid, kPanelThreads, smem, st>>>(g);
    LLS_LAUNCH_CHECK("batched_adjoint", st);
    return LLS_OK;
}

double* batched_adjoint_info_ptr(void* ws, int batch, const int* m, const int* n) {
    ALayout L;
    a_layout(batch, m, n, L);
    return (double*)((char*)ws + L.info);
}

}  // namespace lls
