// Explicit inverse of the upper-triangular R, the preconditioner of the Krylov solve.
//
// Alg. 5 applies R^{-1} and R^{-T} once each per iteration (inv(R)*p, inv(R')*(A'*r)). A
// triangular solve is a chain of n/b dependent steps; with R^{-1} formed once the two
// applications become fully parallel matrix-vector products. Any fixed nonsingular M
// gives a valid preconditioned CGLS as long as the same M is used on both sides, so the
// FP32 rounding of M changes only the convergence rate, not the converged solution.
//
// Formation follows the block structure of Eq. recqr: with R = [R11 R12; 0 R22],
// R^{-1} = [M11, -M11 R12 M22; 0, M22]; leaves (<= 32 columns) are inverted by back
// substitution, one column of the inverse per thread.
#include "common.cuh"
#include "kernels.cuh"

namespace lls {

__global__ void diag_block_inverse_kernel(const float* __restrict__ R, int ldr, int c0, int w,
                                          float* __restrict__ M, int ldm, int* err) {
    __shared__ float Rs[32][33];
    __shared__ float Ms[32][33];
    const int j = threadIdx.x;   // column of the inverse
    for (int i = 0; i < w; ++i)
        Rs[i][j] = (j < w) ? R[(size_t)(c0 + i) + (size_t)(c0 + j) * ldr] : 0.f;
    __syncwarp();
    if (j < w) {
        for (int i = w - 1; i >= 0; --i) {
            float s = (i == j) ? 1.f : 0.f;
            for (int k = i + 1; k <= j; ++k) s = fmaf(-Rs[i][k], Ms[k][j], s);
            float d = Rs[i][i];
            if (!(d != 0.f) || !isfinite(d)) atomicCAS(err, DEV_OK, DEV_SINGULAR);
            Ms[i][j] = (i <= j) ? s / d : 0.f;
        }
    }
    __syncwarp();
    if (j < w)
        for (int i = 0; i < w; ++i) M[(size_t)(c0 + i) + (size_t)(c0 + j) * ldm] = Ms[i][j];
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

static int split_point_host(int w, int pw) { return pw * ceil_div(w, 2 * pw); }

static int inv_rec(const float* R, int ldr, int c0, int w, int pw, float* M, int ldm, float* tmp,
                   int* err, cudaStream_t st) {
    if (w <= pw) {
        diag_block_inverse_kernel<<<1, 32, 0, st>>>(R, ldr, c0, w, M, ldm, err);
        LLS_LAUNCH_CHECK("diag_block_inverse", st);
        return LLS_OK;
    }
    const int w1 = split_point_host(w, pw), w2 = w - w1;
    LLS_TRY(inv_rec(R, ldr, c0, w1, pw, M, ldm, tmp, err, st));
    LLS_TRY(inv_rec(R, ldr, c0 + w1, w2, pw, M, ldm, tmp, err, st));
    // T = R12 M22 (w1 x w2), then M12 = -M11 T
    const float* R12 = R + (size_t)c0 + (size_t)(c0 + w1) * ldr;
    const float* M22 = M + (size_t)(c0 + w1) + (size_t)(c0 + w1) * ldm;
    const float* M11 = M + (size_t)c0 + (size_t)c0 * ldm;
    float* M12 = M + (size_t)c0 + (size_t)(c0 + w1) * ldm;
    LLS_TRY(sgemm(false, false, w1, w2, w2, 1.f, R12, ldr, M22, ldm, 0.f, tmp, w1, st));
    LLS_TRY(sgemm(false, false, w1, w2, w1, -1.f, M11, ldm, tmp, w1, 0.f, M12, ldm, st));
    return LLS_OK;
}

int tri_inverse(const float* R, int ldr, int n, int pw, float* Minv, float* Mt, float* tmp,
                int* dev_err, cudaStream_t st) {
    LLS_CUDA_TRY(cudaMemsetAsync(Minv, 0, sizeof(float) * (size_t)n * n, st));
    LLS_TRY(inv_rec(R, ldr, 0, n, pw < 1 ? 32 : (pw > 32 ? 32 : pw), Minv, n, tmp, dev_err, st));
    if (Mt) {
        dim3 grid(ceil_div(n, 32), ceil_div(n, 32));
        transpose_kernel<<<grid, dim3(32, 8), 0, st>>>(Minv, n, Mt, n, n);
        LLS_LAUNCH_CHECK("transpose", st);
    }
    return LLS_OK;
}

}  // namespace lls
