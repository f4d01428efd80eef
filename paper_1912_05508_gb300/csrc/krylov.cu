// R-preconditioned CGLS (Alg. 5, Sec. 3.2.3) as one persistent cooperative kernel.
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
#include "common.cuh"
#include "kernels.cuh"

namespace lls {

constexpr int kKThreads = 256;
constexpr int kKWarps = kKThreads / 32;
constexpr int kRowTile = 256;     // rows per A t work item (one row per thread)
constexpr int kColChunk = 128;    // columns per A t work item
constexpr int kRowChunk = 2048;   // rows per A^T r work item (staged in shared memory)
constexpr int kColGroup = 32;     // columns per A^T r work item (4 per warp)
constexpr int kMaxRestarts = 3;
constexpr int kNPart = 4;         // block-partial slots

struct KArgs {
    int m, n, lda;
    const float* A;
    const double* b;
    double* x;
    const float* M;
    const float* Mt;
    double *r, *q, *t, *p, *s, *u, *qpart, *upart, *bpart;
    unsigned* bar;
    int* err;
    double* info;
    const double* anorm2;
    const double* mnorm2;
    double tol;
    int max_iter, target, x_zero;
    int nrt, nck, nrc, ncg;
};

extern __shared__ float2 k_dsm[];

__device__ __forceinline__ void stage_vec(const double* __restrict__ v, int len) {
    for (int i = threadIdx.x; i < len; i += kKThreads) {
        float hi, lo;
        split_df(__ldcg(v + i), hi, lo);
        k_dsm[i] = make_float2(hi, lo);
    }
    __syncthreads();
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

// Fixed-order sum of slot k over all blocks (identical in every CTA).
__device__ __forceinline__ double grid_total(const double* bpart, int k) {
    __shared__ double s_tot;
    if (threadIdx.x < 32) {
        double s = 0.0;
        for (int i = threadIdx.x; i < (int)gridDim.x; i += 32) s += __ldcg(bpart + (size_t)k * gridDim.x + i);
        s = warp_sum_d(s);
        if (threadIdx.x == 0) s_tot = s;
    }
    __syncthreads();
    double r = s_tot;
    __syncthreads();
    return r;
}

// out_c = sum over r in [lo(c), hi(c)) of X[r + c n] * v_r, v staged in k_dsm.
// upper: rows 0..c (column c of an upper-triangular X); lower: rows c..n-1.
__device__ double tri_gemv(const float* __restrict__ X, int n, bool upper, double* __restrict__ out) {
    const int lane = threadIdx.x & 31;
    const int gw = blockIdx.x * kKWarps + (threadIdx.x >> 5), nw = gridDim.x * kKWarps;
    double sq = 0.0;
    for (int c = gw; c < n; c += nw) {
        const int lo = upper ? 0 : c, hi = upper ? c + 1 : n;
        const float* col = X + (size_t)c * n;
        float s = 0.f, cc = 0.f;
        for (int r = lo + lane; r < hi; r += 32) {
            float2 v = k_dsm[r];
            dot2_step(s, cc, __ldg(col + r), v.x, v.y);
        }
        double val = warp_sum_d(join_df(s, cc));
        if (lane == 0) { out[c] = val; sq += val * val; }
    }
    return sq;
}

// qpart[cc][i] = sum_{j in chunk cc} A[i, j] * v_j, v staged in k_dsm.
__device__ void a_times_partials(const KArgs& a) {
    const int items = a.nrt * a.nck;
    for (int it = blockIdx.x; it < items; it += gridDim.x) {
        const int rt = it % a.nrt, cc = it / a.nrt;
        const int i = rt * kRowTile + threadIdx.x;
        if (i >= a.m) continue;
        const int j0 = cc * kColChunk, j1 = min(a.n, j0 + kColChunk);
        const float* rowp = a.A + i;
        float s = 0.f, c = 0.f;
#pragma unroll 8
        for (int j = j0; j < j1; ++j) {
            float2 v = k_dsm[j];
            dot2_step(s, c, __ldg(rowp + (size_t)j * a.lda), v.x, v.y);
        }
        a.qpart[(size_t)cc * a.m + i] = join_df(s, c);
    }
}

// upart[rc][j] = sum_{i in row chunk rc} A[i, j] * v_i for v (length m) in global memory.
__device__ void at_times_partials(const KArgs& a, const double* __restrict__ v) {
    const int items = a.nrc * a.ncg;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    for (int it = blockIdx.x; it < items; it += gridDim.x) {
        const int rc = it % a.nrc, cg = it / a.nrc;
        const int r0 = rc * kRowChunk, rows = min(a.m - r0, kRowChunk);
        __syncthreads();
        for (int i = threadIdx.x; i < rows; i += kKThreads) {
            float hi, lo;
            split_df(__ldcg(v + r0 + i), hi, lo);
            k_dsm[i] = make_float2(hi, lo);
        }
        __syncthreads();
        for (int jj = 0; jj < kColGroup / kKWarps; ++jj) {
            const int j = cg * kColGroup + warp * (kColGroup / kKWarps) + jj;
            if (j >= a.n) break;
            const float* col = a.A + (size_t)j * a.lda + r0;
            float s = 0.f, c = 0.f;
#pragma unroll 4
            for (int i = lane; i < rows; i += 32) {
                float2 w = k_dsm[i];
                dot2_step(s, c, __ldg(col + i), w.x, w.y);
            }
            double val = warp_sum_d(join_df(s, c));
            if (lane == 0) a.upart[(size_t)rc * a.n + j] = val;
        }
    }
}

#define KB_SYNC() do { if (!grid_barrier(a.bar, gridDim.x, a.err)) return; } while (0)

__global__ void __launch_bounds__(kKThreads)
cgls_kernel(KArgs a) {
    const int gtid = blockIdx.x * kKThreads + threadIdx.x, gthreads = gridDim.x * kKThreads;
    const double anorm = sqrt(*a.anorm2);
    const double mnorm = sqrt(*a.mnorm2);
    int iters = 0, status = 1, apasses = 0, mpasses = 0;
    double eta = 0.0, fwd = 0.0, rn2 = 0.0, un2 = 0.0, xn2 = 0.0, gamma = 0.0;
    bool xzero = a.x_zero != 0;

    for (int restart = 0; restart <= kMaxRestarts; ++restart) {
        // ---- true residual r = b - A x ----
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
                for (int cc = 0; cc < a.nck; ++cc) ax += __ldcg(a.qpart + (size_t)cc * a.m + i);
                double ri = a.b[i] - ax;
                a.r[i] = ri;
                sq += ri * ri;
            }
            block_partial(sq, a.bpart, 0);
        }
        xzero = false;
        KB_SYNC();
        rn2 = grid_total(a.bpart, 0);
        // ---- u = A^T r, s = M^T u, gamma = ||s||^2 ----
        at_times_partials(a, a.r);
        ++apasses;
        KB_SYNC();
        {
            double sq = 0.0;
            for (int j = gtid; j < a.n; j += gthreads) {
                double v = 0.0;
                for (int rc = 0; rc < a.nrc; ++rc) v += __ldcg(a.upart + (size_t)rc * a.n + j);
                a.u[j] = v;
                sq += v * v;
            }
            block_partial(sq, a.bpart, 1);
            double xs = 0.0;
            for (int j = gtid; j < a.n; j += gthreads) { double xv = __ldcg(a.x + j); xs += xv * xv; }
            block_partial(xs, a.bpart, 3);
        }
        KB_SYNC();
        un2 = grid_total(a.bpart, 1);
        xn2 = grid_total(a.bpart, 3);
        stage_vec(a.u, a.n);
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
        if (crit <= a.tol) { status = 0; break; }
        if (iters >= a.max_iter || restart == kMaxRestarts) { status = 1; break; }
        for (int j = gtid; j < a.n; j += gthreads) a.p[j] = __ldcg(a.s + j);
        KB_SYNC();

        // ---- iterate ----
        bool conv = false;
        while (iters < a.max_iter) {
            // t = M p
            stage_vec(a.p, a.n);
            tri_gemv(a.Mt, a.n, false, a.t);
            ++mpasses;
            KB_SYNC();
            // q = A t, delta = ||q||^2
            stage_vec(a.t, a.n);
            a_times_partials(a);
            ++apasses;
            KB_SYNC();
            {
                double sq = 0.0;
                for (int i = gtid; i < a.m; i += gthreads) {
                    double v = 0.0;
                    for (int cc = 0; cc < a.nck; ++cc) v += __ldcg(a.qpart + (size_t)cc * a.m + i);
                    a.q[i] = v;
                    sq += v * v;
                }
                block_partial(sq, a.bpart, 0);
            }
            KB_SYNC();
            const double delta = grid_total(a.bpart, 0);
            ++iters;
            if (!(delta > 0.0)) { conv = true; break; }
            const double alpha = gamma / delta;
            {
                double xs = 0.0;
                for (int j = gtid; j < a.n; j += gthreads) {
                    double xv = a.x[j] + alpha * __ldcg(a.t + j);
                    a.x[j] = xv;
                    xs += xv * xv;
                }
                block_partial(xs, a.bpart, 3);
                for (int i = gtid; i < a.m; i += gthreads) a.r[i] -= alpha * __ldcg(a.q + i);
            }
            KB_SYNC();
            // s = M^T (A^T r)
            at_times_partials(a, a.r);
            ++apasses;
            KB_SYNC();
            for (int j = gtid; j < a.n; j += gthreads) {
                double v = 0.0;
                for (int rc = 0; rc < a.nrc; ++rc) v += __ldcg(a.upart + (size_t)rc * a.n + j);
                a.u[j] = v;
            }
            KB_SYNC();
            stage_vec(a.u, a.n);
            block_partial(tri_gemv(a.M, a.n, true, a.s), a.bpart, 2);
            ++mpasses;
            KB_SYNC();
            const double gnew = grid_total(a.bpart, 2);
            const double xn = sqrt(grid_total(a.bpart, 3));
            const double beta = gnew / gamma;
            gamma = gnew;
            for (int j = gtid; j < a.n; j += gthreads) a.p[j] = __ldcg(a.s + j) + beta * a.p[j];
            const double sn = sqrt(gnew);
            const double e1 = xn > 0.0 ? sn / (anorm * xn) : INFINITY;
            const double f1 = xn > 0.0 ? mnorm * sn / xn : INFINITY;
            KB_SYNC();
            if ((a.target == LLS_TARGET_FP64 ? e1 : f1) <= a.tol) { conv = true; break; }
        }
        (void)conv;
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
struct KLayout {
    int nrt, nck, nrc, ncg;
    size_t off_r, off_q, off_t, off_p, off_s, off_u, off_qpart, off_upart, off_bpart, off_bar, total;
};

static KLayout k_layout(int m, int n, int grid) {
    KLayout L;
    L.nrt = ceil_div(m, kRowTile);
    L.nck = ceil_div(n, kColChunk);
    L.nrc = ceil_div(m, kRowChunk);
    L.ncg = ceil_div(n, kColGroup);
    size_t o = 0;
    auto take = [&](size_t bytes) { size_t r = o; o = align_up(o + bytes, 256); return r; };
    L.off_r = take(8ull * m);
    L.off_q = take(8ull * m);
    L.off_t = take(8ull * n);
    L.off_p = take(8ull * n);
    L.off_s = take(8ull * n);
    L.off_u = take(8ull * n);
    L.off_qpart = take(8ull * m * L.nck);
    L.off_upart = take(8ull * n * L.nrc);
    L.off_bpart = take(8ull * kNPart * grid);
    L.off_bar = take(64);
    L.total = o;
    return L;
}

size_t krylov_scratch_bytes(int m, int n, int grid) {
    if (grid <= 0) grid = 2 * 160;
    return k_layout(m, n, grid).total;
}

int krylov_solve(const KrylovCall& c, cudaStream_t st) {
    if (c.method != LLS_KRYLOV_CGLS) return LLS_ERR_UNSUPPORTED;
    const size_t smem = sizeof(float2) * (size_t)(c.n > kRowChunk ? c.n : kRowChunk);
    if (smem > 200 * 1024) return LLS_ERR_UNSUPPORTED;
    LLS_CUDA_TRY(cudaFuncSetAttribute(cgls_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    int per_sm = 0;
    LLS_CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, cgls_kernel, kKThreads, smem));
    int dev = 0, sms = 0;
    LLS_CUDA_TRY(cudaGetDevice(&dev));
    LLS_CUDA_TRY(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    if (per_sm < 1) return LLS_ERR_UNSUPPORTED;
    int maxg = sms * (per_sm < 2 ? per_sm : 2);
    // enough CTAs for the work, few enough that barriers stay cheap on small problems
    long long work = (long long)c.m * c.n;
    int grid = (int)((work + (1 << 16) - 1) >> 16);
    if (grid < 1) grid = 1;
    if (grid > maxg) grid = maxg;
    KLayout L = k_layout(c.m, c.n, grid);
    if (L.total > c.scratch_bytes) return LLS_ERR_WORKSPACE;
    char* base = (char*)c.scratch;
    KArgs a;
    a.m = c.m; a.n = c.n; a.lda = c.lda; a.A = c.A; a.b = c.b; a.x = c.x;
    a.M = c.Minv; a.Mt = c.Mt;
    a.r = (double*)(base + L.off_r); a.q = (double*)(base + L.off_q);
    a.t = (double*)(base + L.off_t); a.p = (double*)(base + L.off_p);
    a.s = (double*)(base + L.off_s); a.u = (double*)(base + L.off_u);
    a.qpart = (double*)(base + L.off_qpart); a.upart = (double*)(base + L.off_upart);
    a.bpart = (double*)(base + L.off_bpart);
    a.bar = (unsigned*)(base + L.off_bar);
    a.err = c.dev_err;
    a.info = c.dev_info;
    a.anorm2 = c.dev_info + 8;
    a.mnorm2 = c.dev_info + 9;
    a.tol = c.tol; a.max_iter = c.max_iter; a.target = c.target; a.x_zero = 1;
    a.nrt = L.nrt; a.nck = L.nck; a.nrc = L.nrc; a.ncg = L.ncg;
    LLS_CUDA_TRY(cudaMemsetAsync(a.bar, 0, 64, st));
    void* args[] = {&a};
    LLS_CUDA_TRY(cudaLaunchCooperativeKernel((void*)cgls_kernel, dim3(grid), dim3(kKThreads), args, smem, st));
    note_launch("cgls", st);
    return LLS_OK;
}

}  // namespace lls
