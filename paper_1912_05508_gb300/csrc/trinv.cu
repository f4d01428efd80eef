// Explicit inverse of the upper-triangular R, the preconditioner of the Krylov solve.
//
// Alg. 5 applies R^{-1} and R^{-T} once each per iteration (inv(R)*p, inv(R')*(A'*r)). A
// triangular solve is a chain of n/b dependent steps; with R^{-1} formed once the two
// applications become fully parallel matrix-vector products. Any fixed nonsingular M
// gives a valid preconditioned CGLS as long as the same M is used on both sides, so the
// FP32 rounding of M changes only the convergence rate, not the converged solution.
//
// Formation follows the block structure of Eq. recqr: with R = [R11 R12; 0 R22],
// R^{-1} = [M11, -M11 R12 M22; 0, M22], over the same column split as the QR. All leaves
// (<= 32 columns) are inverted in one launch by back substitution, one column of the
// inverse per thread; the internal nodes of one tree depth are independent and run as
// two batched products per depth, deepest first.
#include <algorithm>
#include <vector>

#include "common.cuh"
#include "kernels.cuh"

namespace lls {

constexpr int kMaxNodes = 1024;

struct NodeList {
    int count;
    int c0[kMaxNodes];
    int w1[kMaxNodes];
    int w2[kMaxNodes];
};

__global__ void diag_block_inverse_kernel(const float* __restrict__ R, int ldr, float* __restrict__ M,
                                          int ldm, int* err, NodeList nl) {
    __shared__ float Rs[32][33];
    __shared__ float Ms[32][33];
    const int c0 = nl.c0[blockIdx.x], w = nl.w1[blockIdx.x];
    const int j = threadIdx.x;   // column of the inverse
    for (int i = 0; i < w; ++i)
        Rs[i][j] = (j < w) ? R[(size_t)(c0 + i) + (size_t)(c0 + j) * ldr] : 0.f;
    __syncwarp();
    if (j < w) {
        for (int i = w - 1; i >= 0; --i) {
            float s = (i == j) ? 1.f : 0.f;
            for (int k = i + 1; k <= j; ++k) s = fmaf(-Rs[i][k], Ms[k][j], s);
            const float d = Rs[i][i];
            if (!(d != 0.f) || !isfinite(d)) atomicCAS(err, DEV_OK, DEV_SINGULAR);
            Ms[i][j] = (i <= j) ? s / d : 0.f;
        }
    }
    __syncwarp();
    if (j < w)
        for (int i = 0; i < w; ++i) M[(size_t)(c0 + i) + (size_t)(c0 + j) * ldm] = Ms[i][j];
}

// One batched product per tree depth, 64 x 64 tiles, FP32. For node (c0, w1, w2):
//   phase 0:  T   = R12 M22      (w1 x w2, K = w2; T stored where M12 will go, in tmp)
//   phase 1:  M12 = -M11 T       (w1 x w2, K = w1)
// M22 and M11 are upper triangular, so the K loop skips their zero blocks. 64 threads per tile,
// each holding 8 x 8 results (rows tx*4 + u and 32 + tx*4 + u, columns likewise with ty), so
// four 16-byte shared reads feed 64 FMAs; every result is one chain of FMAs over k in
// increasing order.
constexpr int kTB = 64, kTK = 16, kTT = 64;
__global__ void __launch_bounds__(kTT)
trinv_batched_kernel(int phase, const float* __restrict__ R, int ldr, float* __restrict__ M,
                     float* __restrict__ tmp, int n, NodeList nl) {
    const int node = blockIdx.z;
    const int c0 = nl.c0[node], w1 = nl.w1[node], w2 = nl.w2[node];
    // a tile's K range grows with j in phase 0 (B = M22 is upper triangular) and shrinks with i
    // in phase 1: the grid is ordered so the longest tiles start first and the short ones fill
    // the last wave
    const int i0 = blockIdx.x * kTB;
    const int j0 = (phase == 0 ? (int)(gridDim.y - 1 - blockIdx.y) : (int)blockIdx.y) * kTB;
    if (i0 >= w1 || j0 >= w2) return;
    const float* A;
    const float* B;
    float* C;
    int lda, ldb, K;
    float alpha;
    if (phase == 0) {
        A = R + (size_t)c0 + (size_t)(c0 + w1) * ldr; lda = ldr;
        B = M + (size_t)(c0 + w1) + (size_t)(c0 + w1) * n; ldb = n;
        C = tmp + (size_t)c0 + (size_t)(c0 + w1) * n;
        K = w2; alpha = 1.f;
    } else {
        A = M + (size_t)c0 + (size_t)c0 * n; lda = n;
        B = tmp + (size_t)c0 + (size_t)(c0 + w1) * n; ldb = n;
        C = M + (size_t)c0 + (size_t)(c0 + w1) * n;
        K = w1; alpha = -1.f;
    }
    // two shared-memory stages: the global loads of step k + 1 are issued into registers
    // before step k's products, so their latency overlaps the arithmetic; one barrier a step
    __shared__ __align__(16) float As[2][kTK][kTB + 4];   // As[k][i]
    __shared__ __align__(16) float Bs[2][kTK][kTB + 4];   // Bs[k][j]
    const int t = threadIdx.x;
    const int tx = t % 8, ty = t / 8;
    float acc[8][8];
#pragma unroll
    for (int u = 0; u < 8; ++u)
#pragma unroll
        for (int v = 0; v < 8; ++v) acc[u][v] = 0.f;
    // phase 0: B = M22 upper triangular, rows k <= j; phase 1: A = M11 upper, columns k >= i
    const int kbeg = phase == 1 ? (i0 / kTK) * kTK : 0;
    const int kend = phase == 0 ? min(K, j0 + kTB) : K;
    float ra[kTK], rb[kTK];
    auto fetch = [&](int k0) {
        const int gi = i0 + t;                            // A: row t of the tile, 16 k
#pragma unroll
        for (int r = 0; r < kTK; ++r) {
            const int gk = k0 + r;
            ra[r] = (gi < w1 && gk < K) ? A[(size_t)gi + (size_t)gk * lda] : 0.f;
        }
        const int kk2 = t % kTK;                          // B: k = t mod 16, columns t / 16 + 4 r
#pragma unroll
        for (int r = 0; r < kTK; ++r) {
            const int gj = j0 + t / kTK + 4 * r, gk2 = k0 + kk2;
            rb[r] = (gj < w2 && gk2 < K) ? B[(size_t)gk2 + (size_t)gj * ldb] : 0.f;
        }
    };
    if (kbeg < kend) fetch(kbeg);
    int stage = 0;
    for (int k0 = kbeg; k0 < kend; k0 += kTK, stage ^= 1) {
#pragma unroll
        for (int r = 0; r < kTK; ++r) {
            As[stage][r][t] = ra[r];
            Bs[stage][t % kTK][t / kTK + 4 * r] = rb[r];
        }
        __syncthreads();
        if (k0 + kTK < kend) fetch(k0 + kTK);
#pragma unroll
        for (int kk = 0; kk < kTK; ++kk) {
            const float4 a0 = *reinterpret_cast<const float4*>(&As[stage][kk][tx * 4]);
            const float4 a1 = *reinterpret_cast<const float4*>(&As[stage][kk][32 + tx * 4]);
            const float4 b0 = *reinterpret_cast<const float4*>(&Bs[stage][kk][ty * 4]);
            const float4 b1 = *reinterpret_cast<const float4*>(&Bs[stage][kk][32 + ty * 4]);
            const float av[8] = {a0.x, a0.y, a0.z, a0.w, a1.x, a1.y, a1.z, a1.w};
            const float bv[8] = {b0.x, b0.y, b0.z, b0.w, b1.x, b1.y, b1.z, b1.w};
#pragma unroll
            for (int u = 0; u < 8; ++u)
#pragma unroll
                for (int v = 0; v < 8; ++v) acc[u][v] = fmaf(av[u], bv[v], acc[u][v]);
        }
    }
#pragma unroll
    for (int v = 0; v < 8; ++v) {
        const int j = j0 + (v < 4 ? ty * 4 + v : 32 + ty * 4 + v - 4);
        if (j >= w2) continue;
#pragma unroll
        for (int u = 0; u < 8; ++u) {
            const int i = i0 + (u < 4 ? tx * 4 + u : 32 + tx * 4 + u - 4);
            if (i < w1) C[(size_t)i + (size_t)j * n] = alpha * acc[u][v];
        }
    }
}

__global__ void transpose_kernel(const float* __restrict__ X, int ldx, float* __restrict__ Y, int ldy, int n) {
    __shared__ float tile[32][33];
    int bx = blockIdx.x * 32, by = blockIdx.y * 32;
    int tx = threadIdx.x, ty = threadIdx.y;
    for (int k = ty; k < 32; k += 8) {
        int r = bx + tx, c = by + k;
        if (r < n && c < n) tile[k][tx] = X[(size_t)r + (size_t)c * ldx];
    }
    __syncthreads();
    for (int k = ty; k < 32; k += 8) {
        int r = by + tx, c = bx + k;
        if (r < n && c < n) Y[(size_t)r + (size_t)c * ldy] = tile[tx][k];
    }
}

// C = U V for upper-triangular U, V: C(i, j) = sum_{k = i..j} U(i, k) V(k, j). 64 x 64 tiles,
// the K loop restricted to [i0, j0 + 64); tiles entirely below the diagonal are written zero.
__global__ void __launch_bounds__(256)
triu_product_kernel(const float* __restrict__ U, int ldu, const float* __restrict__ V, int ldv,
                    float* __restrict__ C, int ldc, int n) {
    const int i0 = blockIdx.x * kTB, j0 = blockIdx.y * kTB;
    __shared__ __align__(16) float As[kTK][kTB + 4];
    __shared__ __align__(16) float Bs[kTK][kTB + 4];
    const int t = threadIdx.x;
    const int ti = (t % 16) * 4, tj = (t / 16) * 4;
    float acc[4][4] = {};
    if (i0 < j0 + kTB) {
        const int kbeg = (i0 / kTK) * kTK, kend = min(n, j0 + kTB);
        for (int k0 = kbeg; k0 < kend; k0 += kTK) {
#pragma unroll
            for (int r = 0; r < 4; ++r) {
                const int idx = t + r * 256;
                const int ii = idx % kTB, kk = idx / kTB;
                const int gi = i0 + ii, gk = k0 + kk;
                As[kk][ii] = (gi < n && gk < n && gk >= gi) ? U[(size_t)gi + (size_t)gk * ldu] : 0.f;
                const int kk2 = idx % kTK, jj = idx / kTK;
                const int gj = j0 + jj, gk2 = k0 + kk2;
                Bs[kk2][jj] = (gj < n && gk2 < n && gk2 <= gj) ? V[(size_t)gk2 + (size_t)gj * ldv] : 0.f;
            }
            __syncthreads();
#pragma unroll
            for (int kk = 0; kk < kTK; ++kk) {
                float av[4], bv[4];
#pragma unroll
                for (int u = 0; u < 4; ++u) { av[u] = As[kk][ti + u]; bv[u] = Bs[kk][tj + u]; }
#pragma unroll
                for (int u = 0; u < 4; ++u)
#pragma unroll
                    for (int v = 0; v < 4; ++v) acc[u][v] = fmaf(av[u], bv[v], acc[u][v]);
            }
            __syncthreads();
        }
    }
#pragma unroll
    for (int v = 0; v < 4; ++v) {
        const int j = j0 + tj + v;
        if (j >= n) continue;
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            const int i = i0 + ti + u;
            if (i < n) C[(size_t)i + (size_t)j * ldc] = i <= j ? acc[u][v] : 0.f;
        }
    }
}

int triu_product(const float* U, int ldu, const float* V, int ldv, float* C, int ldc, int n, cudaStream_t st) {
    dim3 grid(ceil_div(n, kTB), ceil_div(n, kTB));
    triu_product_kernel<<<grid, 256, 0, st>>>(U, ldu, V, ldv, C, ldc, n);
    LLS_LAUNCH_CHECK("triu_product", st);
    return LLS_OK;
}

namespace {
struct TreeNode { int c0, w1, w2, depth; };

int split_point_host(int w, int pw) { return pw * ceil_div(w, 2 * pw); }

void walk(int c0, int w, int pw, int depth, std::vector<TreeNode>& leaves, std::vector<TreeNode>& inner) {
    if (w <= pw) { leaves.push_back({c0, w, 0, depth}); return; }
    const int w1 = split_point_host(w, pw);
    inner.push_back({c0, w1, w - w1, depth});
    walk(c0, w1, pw, depth + 1, leaves, inner);
    walk(c0 + w1, w - w1, pw, depth + 1, leaves, inner);
}

template <typename F>
int for_chunks(const std::vector<TreeNode>& v, F f) {
    for (size_t s = 0; s < v.size(); s += kMaxNodes) {
        NodeList nl;
        nl.count = (int)std::min(v.size() - s, (size_t)kMaxNodes);
        int mw1 = 0, mw2 = 0;
        for (int i = 0; i < nl.count; ++i) {
            nl.c0[i] = v[s + i].c0; nl.w1[i] = v[s + i].w1; nl.w2[i] = v[s + i].w2;
            mw1 = std::max(mw1, nl.w1[i]); mw2 = std::max(mw2, nl.w2[i]);
        }
        LLS_TRY(f(nl, mw1, mw2));
    }
    return LLS_OK;
}
}  // namespace

int tri_inverse(const float* R, int ldr, int n, int pw, float* Minv, float* Mt, float* tmp,
                int* dev_err, cudaStream_t st) {
    pw = pw < 1 ? 32 : (pw > 32 ? 32 : pw);
    std::vector<TreeNode> leaves, inner;
    walk(0, n, pw, 0, leaves, inner);
    LLS_CUDA_TRY(cudaMemsetAsync(Minv, 0, sizeof(float) * (size_t)n * n, st));
    LLS_TRY(for_chunks(leaves, [&](const NodeList& nl, int, int) -> int {
        diag_block_inverse_kernel<<<nl.count, 32, 0, st>>>(R, ldr, Minv, n, dev_err, nl);
        LLS_LAUNCH_CHECK("diag_block_inverse", st);
        return (int)LLS_OK;
    }));
    int maxd = 0;
    for (auto& x : inner) maxd = std::max(maxd, x.depth);
    for (int d = maxd; d >= 0; --d) {
        std::vector<TreeNode> lvl;
        for (auto& x : inner) if (x.depth == d) lvl.push_back(x);
        if (lvl.empty()) continue;
        for (int phase = 0; phase < 2; ++phase) {
            LLS_TRY(for_chunks(lvl, [&](const NodeList& nl, int mw1, int mw2) -> int {
                dim3 grid(ceil_div(mw1, kTB), ceil_div(mw2, kTB), nl.count);
                trinv_batched_kernel<<<grid, kTT, 0, st>>>(phase, R, ldr, Minv, tmp, n, nl);
                LLS_LAUNCH_CHECK("trinv_batched", st);
                return (int)LLS_OK;
            }));
        }
    }
    if (Mt) {
        dim3 grid(ceil_div(n, 32), ceil_div(n, 32));
        transpose_kernel<<<grid, dim3(32, 8), 0, st>>>(Minv, n, Mt, n, n);
        LLS_LAUNCH_CHECK("transpose", st);
    }
    return LLS_OK;
}

}  // namespace lls
