// Plain Householder least squares (Alg. 1, Sec. 3.2.2) on the GPU in FP64 or FP32: the
// comparison solver the mixed-precision method is measured against.
//
// Blocked Householder QR in compact-WY form (the LAPACK geqrf scheme), applied to [A, b] so
// that Q^T b comes out as the last column:
//   for each panel of nb columns starting at j0:
//     panel: for each column j, the reflector H_j = I - tau_j v_j v_j^T (v_j(j) = 1) that
//            maps W(j:m, j) to beta e_1, applied to the rest of the panel. One cooperative
//            launch; every CTA owns fixed rows, and each column needs two grid-wide sums
//            (||x||^2, then v^T W(:, c) for the remaining panel columns) behind bounded
//            grid barriers.
//     T:     the nb x nb upper-triangular factor with H_j0 ... H_j0+nb-1 = I - V T V^T, from
//            G = V^T V:  T_ii = tau_i,  T(0:i, i) = -tau_i T(0:i, 0:i) G(0:i, i).
//     trailing columns (including b):  C <- C - V (T^T (V^T C)), two GEMMs and a TRMM.
//   then x = R^{-1} (Q^T b)(0:n) by triangular solve.
// The panel, the T factor and the copies are this file's kernels; the three dense products
// and the triangular solve of the trailing update are plain library calls (cuBLAS).
#include <cublas_v2.h>

#include <mutex>

#include "common.cuh"
#include "kernels.cuh"

namespace lls {

constexpr int kHhThreads = 256;
constexpr int kHhNb = 32;

template <typename T> __device__ __forceinline__ T hh_sum_warp(T v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(kFullMask, v, o);
    return v;
}

template <typename T>
struct HhArgs {
    T* W; int ldw;          // m x (n + 1) work matrix [A, b]
    T* V; int ldv;          // explicit reflectors of the panel (unit diagonal, zeros above)
    T* tau;                 // nb
    T* part;                // [2][kHhNb + 1][grid] block partials
    unsigned* bar;
    int* err;
    int m, j0, jb;
};

// Block sum of up to `cnt` values per thread (vals), written to part[slot][i][blockIdx.x].
template <typename T>
__device__ void hh_block_partials(const T* vals, int cnt, T* part, int slot) {
    __shared__ T sh[kHhNb + 1][kHhThreads / 32];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    for (int i = 0; i < cnt; ++i) {
        const T s = hh_sum_warp(vals[i]);
        if (lane == 0) sh[i][warp] = s;
    }
    __syncthreads();
    for (int i = threadIdx.x; i < cnt; i += kHhThreads) {
        T t = 0;
        for (int w = 0; w < kHhThreads / 32; ++w) t += sh[i][w];
        part[((size_t)slot * (kHhNb + 1) + i) * gridDim.x + blockIdx.x] = t;
    }
    __syncthreads();
}

// Fixed-order total of partial i of `slot` (identical in every CTA), into smem tot[i].
template <typename T>
__device__ void hh_grid_totals(const T* part, int cnt, int slot, T* tot) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    for (int i = warp; i < cnt; i += kHhThreads / 32) {
        T s = 0;
        for (int b = lane; b < (int)gridDim.x; b += 32)
            s += *((volatile const T*)part + ((size_t)slot * (kHhNb + 1) + i) * gridDim.x + b);
        s = hh_sum_warp(s);
        if (lane == 0) tot[i] = s;
    }
    __syncthreads();
}

#define HH_SYNC() do { if (!grid_barrier(a.bar, gridDim.x, a.err)) return; } while (0)

template <typename T>
__global__ void __launch_bounds__(kHhThreads)
hh_panel_kernel(HhArgs<T> a) {
    __shared__ T tot[kHhNb + 1];
    const int gtid = blockIdx.x * kHhThreads + threadIdx.x, gthreads = gridDim.x * kHhThreads;
    const int m = a.m, j0 = a.j0, jb = a.jb;
    int slot = 0;
    for (int k = 0; k < jb; ++k) {
        const int j = j0 + k;
        T* wj = a.W + (size_t)j * a.ldw;
        // ||W(j+1:m, j)||^2
        // every thread owns the fixed rows j0 + gtid + t * gthreads for the whole panel, so the
        // only value one thread reads from another is the diagonal entry, after a barrier
        T s = 0;
        for (int i = j0 + gtid; i < m; i += gthreads)
            if (i > j) s += wj[i] * wj[i];
        hh_block_partials(&s, 1, a.part, slot);
        HH_SYNC();
        hh_grid_totals(a.part, 1, slot, tot);
        slot ^= 1;
        const T xnorm2 = tot[0];
        const T alpha = wj[j];
        T beta, tauj, scale;
        if (xnorm2 == T(0)) {
            beta = alpha; tauj = 0; scale = 0;
        } else {
            const T nrm = sqrt(alpha * alpha + xnorm2);
            beta = alpha >= T(0) ? -nrm : nrm;
            tauj = (beta - alpha) / beta;
            scale = T(1) / (alpha - beta);
        }
        // v (v_j = 1), written into W below the diagonal and into the explicit V
        T* vk = a.V + (size_t)k * a.ldv - j0;                 // row i of the panel at vk[i]
        for (int i = j0 + gtid; i < m; i += gthreads) {
            T v;
            if (i < j) v = 0;
            else if (i == j) v = 1;
            else { v = wj[i] * scale; wj[i] = v; }
            vk[i] = v;
        }
        // w_c = v^T W(j:m, c) for the remaining panel columns
        const int nc = jb - k - 1;
        T w[kHhNb];
        for (int c = 0; c < nc; ++c) {
            const T* wc = a.W + (size_t)(j + 1 + c) * a.ldw;
            T acc = 0;
            for (int i = j0 + gtid; i < m; i += gthreads)
                if (i >= j) acc += (i == j ? T(1) : wj[i]) * wc[i];
            w[c] = acc;
        }
        hh_block_partials(w, nc, a.part, slot);
        HH_SYNC();
        hh_grid_totals(a.part, nc, slot, tot);
        slot ^= 1;
        for (int c = 0; c < nc; ++c) {
            T* wc = a.W + (size_t)(j + 1 + c) * a.ldw;
            const T f = tauj * tot[c];
            for (int i = j0 + gtid; i < m; i += gthreads)
                if (i >= j) wc[i] -= f * (i == j ? T(1) : wj[i]);
        }
        if (gtid == 0) { wj[j] = beta; a.tau[k] = tauj; }
        // no barrier here: the next column's diagonal entry is read only after its norm
        // barrier, and every other access stays within the owning thread's rows
    }
}

// T factor from G = V^T V (jb x jb, ld jb) and tau, one CTA.
template <typename T>
__global__ void hh_tfactor_kernel(const T* G, const T* tau, T* Tm, int jb) {
    __shared__ T Ts[kHhNb][kHhNb + 1];
    const int t = threadIdx.x;
    for (int i = t; i < kHhNb * kHhNb; i += blockDim.x) Ts[i / kHhNb][i % kHhNb] = 0;
    __syncthreads();
    for (int i = 0; i < jb; ++i) {
        // z = T(0:i, 0:i) G(0:i, i);  T(0:i, i) = -tau_i z;  T_ii = tau_i
        T z = 0;
        if (t < i)
            for (int c = t; c < i; ++c) z += Ts[t][c] * G[c + (size_t)i * jb];
        __syncthreads();
        if (t < i) Ts[t][i] = -tau[i] * z;
        if (t == i) Ts[i][i] = tau[i];
        __syncthreads();
    }
    for (int i = t; i < jb * jb; i += blockDim.x) Tm[(i % jb) + (size_t)(i / jb) * jb] = Ts[i % jb][i / jb];
}

template <typename T>
__global__ void hh_load_kernel(const float* A, int lda, const double* b, T* W, int ldw, int m, int n) {
    const size_t total = (size_t)m * (n + 1);
    for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < total; e += (size_t)gridDim.x * blockDim.x) {
        const int i = (int)(e % m), c = (int)(e / m);
        W[i + (size_t)c * ldw] = c < n ? (T)A[i + (size_t)c * lda] : (T)b[i];
    }
}

template <typename T>
__global__ void hh_store_x_kernel(const T* y, double* x, int n) {
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) x[i] = (double)y[i];
}

template <typename T>
__global__ void hh_copy_kernel(const T* src, T* dst, int n) {
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) dst[i] = src[i];
}

namespace {
struct HhLayout {
    size_t W, V, G, Tm, Wk, Wk2, tau, part, bar, err, y, total;
    int ldw;
};

template <typename T>
HhLayout hh_layout(int m, int n, int grid) {
    HhLayout L;
    L.ldw = (int)align_up((size_t)m, 32);
    size_t o = 0;
    auto take = [&](size_t bytes) { size_t r = o; o = align_up(o + bytes, 256); return r; };
    L.W = take(sizeof(T) * (size_t)L.ldw * (n + 1));
    L.V = take(sizeof(T) * (size_t)m * kHhNb);
    L.G = take(sizeof(T) * kHhNb * kHhNb);
    L.Tm = take(sizeof(T) * kHhNb * kHhNb);
    L.Wk = take(sizeof(T) * (size_t)kHhNb * (n + 1));
    L.Wk2 = take(sizeof(T) * (size_t)kHhNb * (n + 1));
    L.tau = take(sizeof(T) * kHhNb);
    L.part = take(sizeof(T) * 2 * (kHhNb + 1) * (size_t)grid);
    L.bar = take(64);
    L.err = take(64);
    L.y = take(sizeof(T) * (size_t)n);
    L.total = o;
    return L;
}

std::mutex g_cublas_mu;
cublasHandle_t g_cublas[64] = {};

int cublas_for_device(cublasHandle_t* h) {
    int dev = 0;
    LLS_CUDA_TRY(cudaGetDevice(&dev));
    if (dev < 0 || dev >= 64) return LLS_ERR_UNSUPPORTED;
    std::lock_guard<std::mutex> lk(g_cublas_mu);
    if (!g_cublas[dev] && cublasCreate(&g_cublas[dev]) != CUBLAS_STATUS_SUCCESS) return LLS_ERR_CUDA;
    *h = g_cublas[dev];
    return LLS_OK;
}

#define HH_BLAS(call) do { if ((call) != CUBLAS_STATUS_SUCCESS) return LLS_ERR_CUDA; } while (0)

cublasStatus_t gemm(cublasHandle_t h, cublasOperation_t ta, cublasOperation_t tb, int m, int n, int k,
                    double al, const double* A, int lda, const double* B, int ldb, double be, double* C, int ldc) {
    return cublasDgemm(h, ta, tb, m, n, k, &al, A, lda, B, ldb, &be, C, ldc);
}
cublasStatus_t gemm(cublasHandle_t h, cublasOperation_t ta, cublasOperation_t tb, int m, int n, int k,
                    float al, const float* A, int lda, const float* B, int ldb, float be, float* C, int ldc) {
    return cublasSgemm(h, ta, tb, m, n, k, &al, A, lda, B, ldb, &be, C, ldc);
}
cublasStatus_t trmm(cublasHandle_t h, int m, int n, const double* A, int lda, const double* B, int ldb, double* C, int ldc) {
    const double one = 1.0;
    return cublasDtrmm(h, CUBLAS_SIDE_LEFT, CUBLAS_FILL_MODE_UPPER, CUBLAS_OP_T, CUBLAS_DIAG_NON_UNIT, m, n, &one,
                       A, lda, B, ldb, C, ldc);
}
cublasStatus_t trmm(cublasHandle_t h, int m, int n, const float* A, int lda, const float* B, int ldb, float* C, int ldc) {
    const float one = 1.f;
    return cublasStrmm(h, CUBLAS_SIDE_LEFT, CUBLAS_FILL_MODE_UPPER, CUBLAS_OP_T, CUBLAS_DIAG_NON_UNIT, m, n, &one,
                       A, lda, B, ldb, C, ldc);
}
cublasStatus_t trsv(cublasHandle_t h, int n, const double* A, int lda, double* x) {
    return cublasDtrsv(h, CUBLAS_FILL_MODE_UPPER, CUBLAS_OP_N, CUBLAS_DIAG_NON_UNIT, n, A, lda, x, 1);
}
cublasStatus_t trsv(cublasHandle_t h, int n, const float* A, int lda, float* x) {
    return cublasStrsv(h, CUBLAS_FILL_MODE_UPPER, CUBLAS_OP_N, CUBLAS_DIAG_NON_UNIT, n, A, lda, x, 1);
}

int hh_grid(int m) {
    int dev = 0, sms = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
        sms = 148;
    int per = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, hh_panel_kernel<double>, kHhThreads, 0) != cudaSuccess || per < 1)
        per = 1;
    int grid = (m + 4 * kHhThreads - 1) / (4 * kHhThreads);   // at least ~4 rows per thread
    const int cap = sms * (per < 2 ? per : 2);
    return grid < 1 ? 1 : (grid > cap ? cap : grid);
}

template <typename T>
int hh_solve(int m, int n, const float* A, int lda, const double* b, double* x, void* ws, size_t ws_bytes,
             cudaStream_t st) {
    const int grid = hh_grid(m);
    HhLayout L = hh_layout<T>(m, n, grid);
    if (L.total > ws_bytes) return LLS_ERR_WORKSPACE;
    char* base = (char*)ws;
    T* W = (T*)(base + L.W);
    T* V = (T*)(base + L.V);
    T* G = (T*)(base + L.G);
    T* Tm = (T*)(base + L.Tm);
    T* Wk = (T*)(base + L.Wk);
    T* Wk2 = (T*)(base + L.Wk2);
    T* y = (T*)(base + L.y);
    cublasHandle_t h;
    LLS_TRY(cublas_for_device(&h));
    HH_BLAS(cublasSetStream(h, st));
    HH_BLAS(cublasSetPointerMode(h, CUBLAS_POINTER_MODE_HOST));
    LLS_CUDA_TRY(cudaMemsetAsync(base + L.bar, 0, 64, st));
    LLS_CUDA_TRY(cudaMemsetAsync(base + L.err, 0, 64, st));
    hh_load_kernel<T><<<1024, 256, 0, st>>>(A, lda, b, W, L.ldw, m, n);
    LLS_LAUNCH_CHECK("hh_load", st);
    for (int j0 = 0; j0 < n; j0 += kHhNb) {
        const int jb = n - j0 < kHhNb ? n - j0 : kHhNb;
        const int mp = m - j0;
        HhArgs<T> a;
        a.W = W; a.ldw = L.ldw; a.V = V; a.ldv = mp; a.tau = (T*)(base + L.tau); a.part = (T*)(base + L.part);
        a.bar = (unsigned*)(base + L.bar); a.err = (int*)(base + L.err); a.m = m; a.j0 = j0; a.jb = jb;
        void* args[] = {&a};
        LLS_CUDA_TRY(cudaLaunchCooperativeKernel((void*)hh_panel_kernel<T>, dim3(grid), dim3(kHhThreads), args, 0, st));
        LLS_LAUNCH_CHECK("hh_panel", st);
        const int nc = n + 1 - (j0 + jb);          // trailing columns, b included
        // G = V^T V, T factor
        HH_BLAS(gemm(h, CUBLAS_OP_T, CUBLAS_OP_N, jb, jb, mp, T(1), V, mp, V, mp, T(0), G, jb));
        hh_tfactor_kernel<T><<<1, 64, 0, st>>>(G, a.tau, Tm, jb);
        LLS_LAUNCH_CHECK("hh_tfactor", st);
        T* C = W + (size_t)(j0 + jb) * L.ldw + j0;
        HH_BLAS(gemm(h, CUBLAS_OP_T, CUBLAS_OP_N, jb, nc, mp, T(1), V, mp, C, L.ldw, T(0), Wk, jb));
        HH_BLAS(trmm(h, jb, nc, Tm, jb, Wk, jb, Wk2, jb));
        HH_BLAS(gemm(h, CUBLAS_OP_N, CUBLAS_OP_N, mp, nc, jb, T(-1), V, mp, Wk2, jb, T(1), C, L.ldw));
    }
    // y = (Q^T b)(0:n); x = R^{-1} y
    hh_copy_kernel<T><<<(n + 255) / 256, 256, 0, st>>>(W + (size_t)n * L.ldw, y, n);
    LLS_LAUNCH_CHECK("hh_copy", st);
    HH_BLAS(trsv(h, n, W, L.ldw, y));
    hh_store_x_kernel<T><<<(n + 255) / 256, 256, 0, st>>>(y, x, n);
    LLS_LAUNCH_CHECK("hh_store_x", st);
    return LLS_OK;
}
}  // namespace

}  // namespace lls

using namespace lls;

extern "C" size_t lls_householder_workspace_size(int m, int n, int prec) {
    if (n < 1 || m < n) return 0;
    const int grid = hh_grid(m);
    if (prec == LLS_PREC_FP64) return hh_layout<double>(m, n, grid).total;
    if (prec == LLS_PREC_FP32) return hh_layout<float>(m, n, grid).total;
    return 0;
}

extern "C" int lls_householder_solve(int m, int n, int prec, const float* A, int lda, const double* b, double* x,
                                     void* ws, size_t ws_bytes, cudaStream_t stream) {
    if (n < 1 || m < n || lda < m || !A || !b || !x || !ws) return LLS_ERR_ARG;
    if (((uintptr_t)ws & 255) != 0) return LLS_ERR_WORKSPACE;
    if (prec != LLS_PREC_FP64 && prec != LLS_PREC_FP32) return LLS_ERR_ARG;
    if (LLS_DEBUG) lls::debug_reset(stream);
    const int st = prec == LLS_PREC_FP64 ? hh_solve<double>(m, n, A, lda, b, x, ws, ws_bytes, stream)
                                         : hh_solve<float>(m, n, A, lda, b, x, ws, ws_bytes, stream);
    if (!LLS_DEBUG) return st;
    const int d = lls::debug_collect(stream);   // the debug build's index records
    return d != LLS_OK ? d : st;
}
