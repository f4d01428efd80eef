/*
 * lls_gb300.h -- C ABI of the GB300 (sm_103a) mixed-precision QR and least-squares library.
 *
 * Problem (Eq. opt:lls, Sec. 2.2): x* = argmin_x ||A x - b||_2 for a full-column-rank
 * A (m x n, m >= n). Method: a recursive Gram-Schmidt QR (RGSQRF, Alg. 2, Eq. recqr)
 * whose two products per recursion step run on the tensor cores in FP16 / BF16 with
 * FP32 accumulation, a communication-avoiding tall-skinny panel (Eq. caqr) with CGS2
 * leaves, and the resulting R used as a right preconditioner for CGLS (Alg. 5) or
 * LSQR, which recovers FP32- or FP64-level accuracy (Sec. 3.2.3).
 *
 * Conventions for every entry point:
 *  - Matrices are column-major with an explicit leading dimension (ld >= rows).
 *  - Matrix and vector pointers are DEVICE pointers owned by the caller, unless a
 *    parameter says "host". The library never allocates device memory: scratch comes
 *    from the caller's workspace, sized by the matching *_workspace_size query.
 *    Workspace pointers must be 256-byte aligned.
 *  - Work is enqueued on `stream` (0 = legacy default stream). Inputs must not be
 *    modified and outputs not read until the stream reaches that point.
 *  - Return value is a status code (lls_status); no C++ exception crosses the ABI.
 *    Argument errors are detected before anything is enqueued.
 *  - Calls are thread-safe as long as concurrent calls use distinct workspaces.
 */
#ifndef LLS_GB300_H
#define LLS_GB300_H

#include <stddef.h>
#include <cuda_runtime_api.h>

#ifdef __cplusplus
extern "C" {
#endif

/* Status codes. Negative = error (outputs undefined), 0 = success, positive = warning. */
typedef enum {
    LLS_OK = 0,
    LLS_NOT_CONVERGED = 1,     /* iteration limit reached; x holds the last iterate, info filled */
    LLS_ERR_ARG = -1,          /* bad size, leading dimension, null pointer or option value */
    LLS_ERR_SINGULAR = -2,     /* R has a zero or non-finite diagonal entry (rank deficient / inf / nan in A),
                                  or b - A x0 is not finite (inf / nan in b or in a given x0) */
    LLS_ERR_CUDA = -3,         /* a CUDA runtime or driver call failed */
    LLS_ERR_WORKSPACE = -4,    /* workspace too small or misaligned */
    LLS_ERR_TIMEOUT = -5,      /* a bounded device-side wait expired (the kernel returned early) */
    LLS_ERR_UNSUPPORTED = -6,  /* valid but unimplemented option combination */
    LLS_ERR_TOO_LARGE = -7,    /* sizes need more scratch than a fixed-scratch entry point holds */
    LLS_ERR_BOUNDS = -8        /* debug build only: an index check failed and its access was skipped */
} lls_status;

/* Precision of the two tensor-core products of each recursion step (Alg. 2: projection and update).
 * FP16 is the paper's choice (Sec. 2.1); BF16 trades resolution for range; FP8 is E4M3 with a
 * power-of-two scale per column of both operands (max in [2^7, 2^8)), 3 significand bits
 * (requires panel_width 16 or 32); FP32 runs the products on the FP32 units (no rounding of
 * the inputs), a reference mode. FP64 is used only by the plain Householder solver below. */
typedef enum { LLS_PREC_FP16 = 0, LLS_PREC_BF16 = 1, LLS_PREC_FP8 = 2, LLS_PREC_FP32 = 3, LLS_PREC_FP64 = 4 } lls_gemm_prec;

/* Accuracy target of the Krylov refinement (Sec. 3.2.3). */
typedef enum { LLS_TARGET_FP32 = 0, LLS_TARGET_FP64 = 1 } lls_target;

/* Krylov method: CGLS (Alg. 5) or LSQR (Paige-Saunders; named in Sec. 5). */
typedef enum { LLS_KRYLOV_CGLS = 0, LLS_KRYLOV_LSQR = 1 } lls_krylov;

/* Starting point of the Krylov iteration. Alg. 5 starts from x = 0 (LLS_X0_ZERO). LLS_X0_GIVEN
 * starts from the x the caller passes in (a warm start, e.g. the solution of a nearby problem).
 * LLS_X0_DIRECT starts from the direct solve with the mixed-precision factors,
 * x0 = R^{-1} (Q^T b) (Alg. 1's last two steps on the RGSQRF Q and R; Sec. 3.2.2 and 4.2.2):
 * its error is at the level of the low-precision products, so CGLS starts with
 * ||A (x0 - x*)|| of about u_low ||b|| instead of ||b|| and needs fewer iterations. */
typedef enum { LLS_X0_ZERO = 0, LLS_X0_GIVEN = 1, LLS_X0_DIRECT = 2 } lls_x0;

typedef struct {
    int gemm_prec;     /* lls_gemm_prec, default LLS_PREC_FP16 */
    int target;        /* lls_target, default LLS_TARGET_FP64 */
    double tol;        /* stop tolerance; <= 0 selects the target's default:
                          FP64: eta_est = ||R^-T A^T r|| / (||A||_F ||x||) <= 1e-12
                          FP32: fwd_est = ||R^-1||_F ||R^-T A^T r|| / ||x|| <= 1e-6 */
    int max_iter;      /* iteration cap, default 200 (the paper's cap, Sec. 4.2.3) */
    int panel_width;   /* recursion leaf width b (columns per panel), 1..32; 0 = auto: the setting
                          recorded by lls_autotune for the shape, else 16 (the paper uses 32,
                          Sec. 3.1.3) */
    int krylov;        /* lls_krylov, default CGLS */
    int leaf_rows;     /* reserved, 0 or 256 (the GPU panel's CAQR row blocks are 1024 rows, Sec. 3.1.3) */
    int reorth;        /* 1: re-orthogonalize (Sec. 4.2.1): factor Q once more, Q1 = Q2 R2, and return
                          Q2 and R = R2 R1 (twice the QR cost); 0 (default): one pass */
    int panel_leaf;    /* leaf factorization of the CAQR panel: 0 (default) CGS2, classical
                          Gram-Schmidt with one reorthogonalization; 1 MGS, the paper's modified
                          Gram-Schmidt leaf (Alg. 4), which loses orthogonality in proportion to the
                          panel's condition number. MGS panels are built for panels whose stacked
                          leaf R factors fit one level (m <= 65536 at panel_width 16); taller panels,
                          and the batched solver, return LLS_ERR_UNSUPPORTED with it. */
    int x0;            /* lls_x0, default LLS_X0_ZERO; the batched solver takes LLS_X0_ZERO only */
} lls_options;

typedef struct {
    int status;        /* lls_status of the call */
    int iters;         /* Krylov iterations performed */
    double eta;        /* eta_est of the returned x, from a freshly computed residual b - A x */
    double fwd_est;    /* ||R^-1||_F ||R^-T A^T r|| / ||x||: estimated relative forward error bound */
    double res_norm;   /* ||b - A x||_2 */
    double atr_norm;   /* ||A^T (b - A x)||_2 */
    double anorm_f;    /* ||A||_F */
    double xnorm;      /* ||x||_2 */
    float qr_ms;       /* device time of the factorization (and preconditioner set-up) */
    float krylov_ms;   /* device time of the Krylov iteration */
    int a_passes;      /* full passes over A made by the Krylov phase (A x, A^T r products; the
                          one-pass CGLS engine's row-block copy of A counts as 2: read + write) */
    int m_passes;      /* products with the n x n preconditioner R^{-1} or its transpose */
} lls_info;

/* Fill *opts with the defaults listed above. */
void lls_default_options(lls_options* opts);

/* Human-readable name of a status code (static string). */
const char* lls_status_string(int status);

/* Number of GPU kernels this process has enqueued through the library so far (all
 * threads, all devices). Lets a caller count launches per call or per captured graph. */
unsigned long long lls_kernel_launch_count(void);

/* ---------------------------------------------------------------------------
 * QR factorization (Alg. 2 + Eq. caqr): A = Q R, Q m x n with orthonormal columns
 * (to the GEMM precision), R n x n upper triangular with positive diagonal.
 *
 *  A  [in]  m x n FP32, lda >= m. Not modified.
 *  Q  [out] m x n FP32, ldq >= m, or NULL when Q is not wanted.
 *  R  [out] n x n FP32, ldr >= n; the strictly lower triangle is set to zero.
 *  ws [in]  workspace of ws_bytes >= qr_factor_workspace_size(m, n, opts), 256-B aligned.
 *  opts     may be NULL (defaults). Only gemm_prec, panel_width and leaf_rows are used.
 * Errors: LLS_ERR_ARG (n < 1, m < n, ld too small, null A/R/ws), LLS_ERR_WORKSPACE,
 *         LLS_ERR_UNSUPPORTED, LLS_ERR_CUDA. Rank deficiency is not an error here:
 *         it shows up as a zero diagonal entry of R. The call does not synchronize, so a
 *         device-side failure (a bounded wait that gave up) cannot be returned: it leaves
 *         NaN on the whole diagonal of R instead.
 * -------------------------------------------------------------------------- */
size_t qr_factor_workspace_size(int m, int n, const lls_options* opts);
int qr_factor(int m, int n, const float* A, int lda, float* Q, int ldq, float* R, int ldr,
              void* ws, size_t ws_bytes, const lls_options* opts, cudaStream_t stream);

/* ---------------------------------------------------------------------------
 * Least-squares solve (Alg. 5 with the QR above as right preconditioner).
 * opts->krylov selects the iteration on the preconditioned operator A R^{-1}: CGLS
 * (Alg. 5, default) or LSQR (Golub-Kahan bidiagonalization, Paige-Saunders; Sec. 5).
 * Both stop on the same tests (lls_options.tol) and confirm them on a fresh residual.
 *
 *  A     [in]  m x n FP32, lda >= m; the problem is defined for these FP32 values.
 *  b     [in]  m FP64.
 *  x     [out] n FP64 (the FP32 target also returns FP64); [in] as well with
 *              opts->x0 = LLS_X0_GIVEN, where it holds the starting point.
 *  R_out [out] n x n FP32 (ldr >= n) receives the preconditioner R, or NULL.
 *  info  [out] HOST pointer or NULL. When non-NULL the call synchronizes `stream`
 *              before returning and fills *info; when NULL the call is fully
 *              asynchronous (and can be captured in a CUDA graph) and the status
 *              returned covers argument checks and launches only.
 * Errors: as qr_factor, plus LLS_ERR_SINGULAR, LLS_ERR_TIMEOUT (reported only through
 *         info), LLS_NOT_CONVERGED (warning).
 * -------------------------------------------------------------------------- */
size_t lls_solve_workspace_size(int m, int n, const lls_options* opts);
int lls_solve(int m, int n, const float* A, int lda, const double* b, double* x,
              float* R_out, int ldr, void* ws, size_t ws_bytes, const lls_options* opts,
              lls_info* info, cudaStream_t stream);

/* ---------------------------------------------------------------------------
 * lls_solve_host: lls_solve on operands that live in page-locked HOST memory (allocated
 * with cudaHostAlloc / cudaMallocHost or registered with cudaHostRegister). The library has
 * no counterpart in the paper; it exists so that a caller whose data is on the host pays for
 * the upload only once, overlapped with the factorization: A is copied up in column chunks of
 * doubling width (64, 64, 128, 256, ... columns) on a library-owned side stream, and the
 * recursion of Alg. 2 waits for a chunk just before it first touches the chunk's columns
 * (columns are first touched in increasing order). x is copied back at the end of the same
 * stream order.
 *  A  [in]  m x n FP32 page-locked host memory, column-major, lda >= m.
 *  b  [in]  m FP64 page-locked host memory.
 *  x  [out] n FP64 page-locked host memory; valid once `stream` has synchronized (the call
 *           synchronizes itself when info is non-NULL). [in] as well with opts->x0 =
 *           LLS_X0_GIVEN: it is uploaded with b and is the starting point.
 *  ws       lls_solve_host_workspace_size(m, n, opts) bytes of DEVICE memory, 256-B
 *           aligned: the lls_solve workspace plus device copies of A, b and x.
 *  opts, info, stream: as lls_solve (no R_out).
 * Errors: as lls_solve; LLS_ERR_ARG also when A, b or x is not page-locked host memory.
 * -------------------------------------------------------------------------- */
size_t lls_solve_host_workspace_size(int m, int n, const lls_options* opts);
/* The column chunks of lls_solve_host's upload for n columns: writes start[0..count] (chunk k
 * covers columns [start[k], start[k+1]), start[0] = 0, start[count] = n) and returns count, or
 * LLS_ERR_ARG (n < 1, start NULL, max_entries < count + 1). Host only. */
int lls_upload_chunks(int n, int* start, int max_entries);
int lls_solve_host(int m, int n, const float* A, int lda, const double* b, double* x, void* ws,
                   size_t ws_bytes, const lls_options* opts, lls_info* info, cudaStream_t stream);

/* ---------------------------------------------------------------------------
 * Batched solve: `batch` independent problems min ||A_i x_i - b_i||, uneven sizes, in one
 * persistent launch (each SM takes whole problems from a device work queue, largest first,
 * and runs factorization, preconditioner and CGLS on its own; 16-column panels).
 *  m, n, lda, ldr: HOST arrays of `batch` ints; n_i <= m_i <= 8192, n_i <= 1024.
 *  A, b, x, R_out: HOST arrays of `batch` DEVICE pointers (A_i m_i x n_i FP32, b_i m_i FP64,
 *     x_i n_i FP64 output, R_out_i n_i x n_i FP32 output or NULL; R_out itself may be NULL).
 *  ws: lls_solve_batched_workspace_size(batch, m, n, opts) bytes, 256-byte aligned.
 *  infos: HOST array of `batch` lls_info, or NULL. When non-NULL the call synchronizes the
 *     stream and fills one record per problem (krylov_ms holds the whole batch's time);
 *     the return value is then the worst per-problem status.
 *  opts: gemm_prec FP16 or BF16; panel_width is fixed at 16 in this path.
 * The problem table is copied into the workspace first; the launch itself is replayed as
 * a CUDA graph on non-default streams.
 * Errors: LLS_ERR_ARG, LLS_ERR_WORKSPACE, LLS_ERR_UNSUPPORTED (sizes, FP32 products, LSQR),
 *         LLS_ERR_CUDA; per-problem LLS_ERR_SINGULAR / LLS_NOT_CONVERGED through infos.
 * -------------------------------------------------------------------------- */
size_t lls_solve_batched_workspace_size(int batch, const int* m, const int* n, const lls_options* opts);
int lls_solve_batched(int batch, const int* m, const int* n, const float* const* A, const int* lda,
                      const double* const* b, double* const* x, float* const* R_out, const int* ldr,
                      void* ws, size_t ws_bytes, const lls_options* opts, lls_info* infos,
                      cudaStream_t stream);

/* ---------------------------------------------------------------------------
 * Adjoint of the least-squares solution map (the paper has none; this is the textbook
 * sensitivity of x* = (A^T A)^{-1} A^T b, used by the differentiable solve).
 * For each problem i of the batch, given x_i = x*(A_i, b_i), the R factor R_i returned by
 * lls_solve (R_out) and g_i = dL/dx_i:
 *     z = (A^T A)^{-1} g   by CG on A^T A z = g preconditioned with (R^T R)^{-1}
 *     grad_b = A z,   grad_A = (b - A x) z^T - (A z) x^T
 *  m, n, lda, ldr, ldga: HOST arrays of `batch` ints (ldr >= n, lda, ldga >= m).
 *  A, b, x, R, grad_x, grad_A, grad_b: HOST arrays of `batch` DEVICE pointers:
 *     A m x n FP32, b m FP64, x n FP64, R n x n FP32 upper triangular, grad_x n FP64,
 *     grad_A m x n FP32 (written), grad_b m FP64 (written).
 *  ws: lls_backward_workspace_size(batch, m, n, opts) bytes, 256-byte aligned.
 *  opts: target FP64 iterates z to ||R^-T (g - A^T A z)|| <= 1e-13 ||R^-T g|| (FP32: 1e-7);
 *        max_iter caps the CG iterations.
 * A batch of two or more problems that the batched solver takes (n_i <= m_i <= 8192,
 * n_i <= 1024) runs as one persistent launch in which each CTA takes whole problems from a
 * work queue (R^{-1}, CG and the gradient on one SM, compensated products as in the solve);
 * a single problem, or a batch with a larger one, runs problem after problem on the whole GPU.
 * Errors: LLS_ERR_ARG, LLS_ERR_WORKSPACE, LLS_ERR_UNSUPPORTED, LLS_ERR_CUDA.
 * -------------------------------------------------------------------------- */
size_t lls_backward_workspace_size(int batch, const int* m, const int* n, const lls_options* opts);
int lls_backward(int batch, const int* m, const int* n, const float* const* A, const int* lda,
                 const double* const* b, const double* const* x, const float* const* R, const int* ldr,
                 const double* const* grad_x, float* const* grad_A, const int* ldga,
                 double* const* grad_b, void* ws, size_t ws_bytes, const lls_options* opts,
                 cudaStream_t stream);

/* ---------------------------------------------------------------------------
 * Kernel-level building blocks: the two tensor-core products of one recursion step of
 * Alg. 2 (projection R12 = Q1^T A2, update A2 = A2 - Q1 R12), with the operands already
 * rounded to FP16 or BF16 (prec = LLS_PREC_FP16 / LLS_PREC_BF16) and FP32 accumulation.
 * Exposed for testing and for callers that run their own recursion.
 *
 * lls_lowp_projection:
 *   Q1l  [in]  m x w1 low-precision, column-major, ldh >= m (ldh * 2 bytes multiple of 16,
 *              base 16-byte aligned); A2l [in] m x w2 low-precision, same ldh.
 *   e    [in]  w2 ints: A2l column j holds A2[:, j] * 2^e[j].
 *   R12  [out] w1 x w2 FP32 (ldr >= w1): (Q1l^T A2l)[:, j] * 2^-e[j], summed in a fixed order.
 *   R12l [out] w1 x w2 low-precision (ldrl >= w1, multiple of 8): R12[:, j] * 2^f[j] rounded
 *              to nearest even, f [out] w2 ints chosen so max|R12[:, j]| 2^f[j] lies in
 *              [2^14, 2^15) for FP16 (f = 0 for BF16).
 *   ws        workspace of lls_lowp_projection_workspace_size(m, w1, w2) bytes, 256-B aligned.
 * lls_lowp_update:
 *   A2 [in/out] m x w2 FP32 (lda >= m): A2 -= (Q1l R12l)[:, j] * 2^-f[j].
 *   ws          >= 256 bytes of 256-B aligned scratch (device error word).
 * Both calls are asynchronous, so a failure on the device cannot be returned: if a bounded
 * device wait gives up (about 2 s), the affected outputs are written as NaN instead (the whole
 * of R12 and R12l with f = 0 for the projection; the affected 128-row tiles of A2 for the
 * update), and the error word in ws holds LLS_ERR_TIMEOUT's device code.
 * Errors: LLS_ERR_ARG, LLS_ERR_WORKSPACE, LLS_ERR_UNSUPPORTED (alignment), LLS_ERR_CUDA.
 * -------------------------------------------------------------------------- */
size_t lls_lowp_projection_workspace_size(int m, int w1, int w2);
int lls_lowp_projection(int m, int w1, int w2, int prec, const void* Q1l, const void* A2l, int ldh,
                        const int* e, float* R12, int ldr, void* R12l, int ldrl, int* f,
                        void* ws, size_t ws_bytes, cudaStream_t stream);
int lls_lowp_update(int m, int w1, int w2, int prec, const void* Q1l, int ldh, const void* R12l,
                    int ldrl, const int* f, float* A2, int lda, void* ws, size_t ws_bytes,
                    cudaStream_t stream);

/* ---------------------------------------------------------------------------
 * lls_panel_qr: the tall-skinny panel factorization of one recursion leaf (Eq. caqr,
 * Sec. 3.1.3): communication-avoiding QR over row blocks of <= 1024 rows with CGS2 leaves
 * (classical Gram-Schmidt with one reorthogonalization; the paper's leaf is MGS, Alg. 4),
 * the b x b R factors combined up a reduction tree, and each block's Q multiplied by its
 * path of tree Q factors. Exposed for testing and for callers that run their own recursion.
 *   m >= b, 1 <= b <= 32.
 *   W   [in/out] m x b FP32, column-major (ldw >= m): the panel in, Q (orthonormal columns) out.
 *   Wh  [out]    m x b copy of Q rounded to nearest even to FP16/BF16 (ldh >= m); ignored and
 *                may be NULL when prec = LLS_PREC_FP32.
 *   R   [out]    b x b upper triangular FP32 (ldr >= b) with a nonnegative diagonal; the
 *                strict lower triangle is written with zeros. A = Q R.
 *   ws           lls_panel_qr_workspace_size(m, b) bytes, 256-B aligned (tree buffers,
 *                arrival counters, device error word). Zero-fill it once before its first
 *                use: every call leaves the counters at zero again, so back-to-back calls on
 *                one stream reuse it without clearing (calls that overlap on the GPU race).
 * Asynchronous on `stream`; no host synchronisation. The one-launch path waits (bounded,
 * about 2 s) for co-resident CTAs; if such a wait gives up, Q and R are undefined and the
 * error word stays set, so the workspace must be zero-filled again before the next call.
 * Errors: LLS_ERR_ARG, LLS_ERR_WORKSPACE, LLS_ERR_UNSUPPORTED, LLS_ERR_CUDA.
 * -------------------------------------------------------------------------- */
size_t lls_panel_qr_workspace_size(int m, int b);
int lls_panel_qr(int m, int b, int prec, float* W, int ldw, void* Wh, int ldh, float* R, int ldr,
                 void* ws, size_t ws_bytes, cudaStream_t stream);

/* ---------------------------------------------------------------------------
 * lls_panel_block_qr: the lowest node of the recursion (Alg. 2) in one launch: the panel of
 * columns [0, w1) (as lls_panel_qr), the node's projection R12 = Q1^T A2 and update
 * A2 = A2 - Q1 R12 with FP16/BF16 operands, FP32 accumulation and the power-of-two column
 * scaling of Sec. 3.1.2, then the panel of columns [w1, w1 + w2). Exposed for testing and for
 * callers that run their own recursion.
 *   8 < w1 <= 16, 1 <= w2 <= w1, m >= w1 + w2; prec = LLS_PREC_FP16 or LLS_PREC_BF16.
 *   W   [in/out] m x (w1 + w2) FP32, column-major (ldw >= m): A in, Q out.
 *   Wh  [out]    m x (w1 + w2) copy of Q rounded to nearest even to prec (ldh >= m).
 *   R   [out]    (w1 + w2) x (w1 + w2) upper triangular FP32 (ldr >= w1 + w2): R11, R12 and
 *                R22 of A = Q R; the strict lower triangle is written with zeros.
 *   ws           lls_panel_block_qr_workspace_size(m, w1, w2) bytes, 256-B aligned. Zero-fill
 *                it once before its first use: every call leaves it ready for the next call
 *                on the same stream (calls that overlap on the GPU race).
 * Asynchronous on `stream`. All CTAs must be co-resident (cooperative launch); each grid
 * wait is bounded (about 2 s) and, if it gives up, Q and R are undefined, the call's error
 * word stays set and the workspace must be zero-filled again.
 * Errors: LLS_ERR_ARG, LLS_ERR_WORKSPACE, LLS_ERR_CUDA; LLS_ERR_UNSUPPORTED (nothing launched)
 * when m is beyond the one-level panel (m > 65536) or w1, w2 are outside the range above.
 * -------------------------------------------------------------------------- */
size_t lls_panel_block_qr_workspace_size(int m, int w1, int w2);
int lls_panel_block_qr(int m, int w1, int w2, int prec, float* W, int ldw, void* Wh, int ldh, float* R,
                       int ldr, void* ws, size_t ws_bytes, cudaStream_t stream);

/* ---------------------------------------------------------------------------
 * Autotuning. The paper picks its panel size by hand for its GPU (Sec. 3.1.3, 256 x 32 blocks
 * on a V100); here the implementation choices are measured per problem shape on the GPU in use
 * and the fastest is recorded. A recorded setting is used by every later call on the same
 * device with the same shape and the same gemm_prec, target, krylov, reorth and panel_leaf
 * whose opts->panel_width is 0 ("auto"; a NULL opts counts as auto). Calls with an explicit
 * panel_width use the library's defaults for the other choices. None of the choices changes the
 * definition of the arithmetic: every kernel keeps its rounding points and summation order.
 * The table lives in the process; lls_tuning_get / lls_tuning_set let a caller save it and
 * restore it (the Python binding keeps a JSON cache this way).
 *
 * lls_tuning (one recorded setting):
 *   panel_width          leaf width b of the recursion (8, 16 or 32);
 *   node_mode            0: the lowest nodes with both of their panels, and the narrow nodes
 *                        (w1 <= 32), each as one launch; 1: narrow nodes as one launch, panels
 *                        separate; 2: every node as four launches (cast, projection, reduction,
 *                        update);
 *   gemm_kernel          products of the wide nodes: 0 persistent (one CTA per SM looping over
 *                        tiles, two accumulators), 1 one output tile per CTA, 2 the persistent
 *                        update with the one-tile-per-CTA projection;
 *   batched_ctas_per_sm  batched solver: CTAs per SM (0 = as many as fit);
 *   krylov_ctas          CTAs of the Krylov kernel (0 = one per 64 Ki elements of A, at most
 *                        three per SM; small problems may run faster on more);
 *   ms                   the measured device time of one call with this setting.
 *
 * lls_autotune: times lls_solve on the caller's problem (A m x n FP32 lda >= m, b m FP64, x n
 *   FP64 output, all device memory) for panel widths 8 / 16 / 32, then the node launch modes,
 *   then the product kernel, then (when the problem would use fewer CTAs than SMs) wider
 *   Krylov grids (coordinate search; each candidate: one untimed call, then the
 *   fastest of `reps`), records the fastest for (m, n, opts) and returns it in *best. opts as
 *   for lls_solve (opts->panel_width is ignored; x0 = LLS_X0_GIVEN is rejected). ws: at least
 *   lls_autotune_workspace_size(m, n, opts) bytes. Synchronizes `stream`. x receives the last
 *   trial's solution.
 * lls_autotune_batched: the same for lls_solve_batched over its CTAs per SM (1 to 4, capped by
 *   what fits); arguments as lls_solve_batched (no R_out), the setting is recorded for the key
 *   (kind 1, m = batch, n = the largest n_i).
 * lls_tuning_set / lls_tuning_get: record / read the setting of a key; kind 0 = lls_solve,
 *   lls_solve_host and qr_factor on m x n; kind 1 = lls_solve_batched (m = batch, n = the
 *   largest n_i). get returns 1 when a setting is recorded, 0 when not. lls_tuning_clear
 *   forgets every recorded setting.
 * Errors: LLS_ERR_ARG, LLS_ERR_WORKSPACE, LLS_ERR_UNSUPPORTED (no candidate ran), LLS_ERR_CUDA.
 * -------------------------------------------------------------------------- */
typedef struct {
    int panel_width;
    int node_mode;
    int gemm_kernel;
    int batched_ctas_per_sm;
    int krylov_ctas;
    float ms;
} lls_tuning;
size_t lls_autotune_workspace_size(int m, int n, const lls_options* opts);
int lls_autotune(int m, int n, const float* A, int lda, const double* b, double* x, void* ws, size_t ws_bytes,
                 const lls_options* opts, int reps, lls_tuning* best, cudaStream_t stream);
int lls_autotune_batched(int batch, const int* m, const int* n, const float* const* A, const int* lda,
                         const double* const* b, double* const* x, void* ws, size_t ws_bytes,
                         const lls_options* opts, int reps, lls_tuning* best, cudaStream_t stream);
int lls_tuning_set(int kind, int m, int n, const lls_options* opts, const lls_tuning* t);
int lls_tuning_get(int kind, int m, int n, const lls_options* opts, lls_tuning* t);
void lls_tuning_clear(void);

/* ---------------------------------------------------------------------------
 * lls_selftest_wait_timeout: exercises the failure path of the library's bounded device
 * waits (no counterpart in the paper). It launches a two-CTA cooperative kernel whose grid
 * barrier expects three arrivals, so the barrier can never complete; each wait gives up after
 * its time limit (about 2 s), sets the device error word and returns. Nothing faults, and the
 * context stays usable.
 *  ws: at least 256 bytes of device memory, 256-B aligned (the barrier words and error word).
 * Synchronizes `stream`. Returns LLS_ERR_TIMEOUT when the wait ran out as designed, LLS_OK if
 * the barrier completed (a defect), LLS_ERR_ARG or LLS_ERR_CUDA otherwise.
 * -------------------------------------------------------------------------- */
int lls_selftest_wait_timeout(void* ws, size_t ws_bytes, cudaStream_t stream);

/* ---------------------------------------------------------------------------
 * Debug build (no counterpart in the paper). The library also builds as
 * liblls_gb300_debug.so, with the same ABI, where the kernels' global-memory accesses carry
 * index checks: a failed check skips its access and records its source line. The compute
 * entry points (qr_factor, lls_solve, lls_solve_host, lls_solve_batched, lls_backward,
 * lls_panel_qr, lls_panel_block_qr, lls_lowp_projection, lls_lowp_update,
 * lls_householder_solve) clear the records before the work, synchronize `stream` after it
 * and return LLS_ERR_BOUNDS (naming the file and line on stderr) if a check failed; debug
 * calls therefore cannot be captured into a caller's CUDA graph. The checks do not change
 * the arithmetic: the two builds give bitwise equal results.
 * lls_debug_build: 1 in the debug build, 0 in the release build.
 * lls_debug_inject: arms a planted fault of the one-level CAQR panel kernels (which factor the
 *   panels of up to 65536 rows), for tests of the failure paths, or disarms it (mode 0):
 *   mode 1: every store of Q is addressed one panel height past the last row; the index
 *           checks reject each such store, so none happens and Q keeps its previous contents;
 *           the call returns LLS_ERR_BOUNDS;
 *   mode 2: the grid barrier between the leaves and the tree waits for one CTA more than the
 *           grid holds; each CTA's bounded wait gives up after about 2 s and sets the device
 *           error word, and the kernels after it return at their first wait: lls_solve returns
 *           LLS_ERR_TIMEOUT, qr_factor leaves NaN on the diagonal of R.
 *   Nothing faults in either mode. Returns LLS_OK, LLS_ERR_ARG (mode not 0, 1 or 2),
 *   LLS_ERR_UNSUPPORTED in the release build, LLS_ERR_CUDA if the flag could not be set.
 * -------------------------------------------------------------------------- */
int lls_debug_build(void);
int lls_debug_inject(int mode);

/* ---------------------------------------------------------------------------
 * Plain Householder least squares (Alg. 1, Sec. 3.2.2): the comparison solver the
 * mixed-precision method is measured against, in FP64 (prec = LLS_PREC_FP64) or FP32
 * (LLS_PREC_FP32) arithmetic throughout. Blocked Householder QR of [A, b] in compact-WY
 * form (32-column panels factored by a cooperative kernel; the trailing update
 * C -= V T^T V^T C and the final triangular solve through cuBLAS), then x = R^{-1} (Q^T b).
 *  A [in] m x n FP32 (lda >= m), b [in] m FP64, x [out] n FP64 (rounded from the working
 *  precision); ws: lls_householder_workspace_size(m, n, prec) bytes, 256-B aligned.
 * Asynchronous on `stream`. No rank check: a zero pivot gives inf/nan in x.
 * Errors: LLS_ERR_ARG (n < 1, m < n, lda < m, null pointers, prec), LLS_ERR_WORKSPACE,
 *         LLS_ERR_UNSUPPORTED, LLS_ERR_CUDA.
 * -------------------------------------------------------------------------- */
size_t lls_householder_workspace_size(int m, int n, int prec);
int lls_householder_solve(int m, int n, int prec, const float* A, int lda, const double* b, double* x,
                          void* ws, size_t ws_bytes, cudaStream_t stream);

/* ---------------------------------------------------------------------------
 * lls_lowp_projection_noalloc: lls_lowp_projection without a workspace argument. The paper
 * has no counterpart; this entry point exists for callers that cannot allocate device memory
 * when they need the product, e.g. code inside a framework's op or plugin hook whose memory
 * pool forbids allocation during execution, latency-bound paths that cannot afford the
 * implicit device synchronisation of cudaMalloc/cudaFree, or host code that only holds
 * borrowed device pointers. It allocates nothing: no cudaMalloc, cudaFree or allocating
 * library routine. Its scratch (split-K partial sums and a device error word) is one
 * file-scope device array of LLS_NOALLOC_SCRATCH_BYTES (4 MiB) inside the library, which
 * every GPU that loads the library holds until the process exits.
 *
 * Arguments, layouts, outputs and the order of summation are those of lls_lowp_projection;
 * Q1l, A2l, e, R12, R12l and f are caller-owned device memory, as there.
 * Limit: accepted when lls_lowp_projection_workspace_size(m, w1, w2) <= LLS_NOALLOC_SCRATCH_BYTES,
 *   otherwise LLS_ERR_TOO_LARGE is returned before any work (for example m = 8192 with
 *   w1 = w2 = 128 fits; m = 32768 with w1 = w2 = 256 does not).
 * Set-up: the first call on each device, with that device current, looks up the array's
 *   device address (cudaGetSymbolAddress) and caches it; make that first call before any
 *   stream capture begins. cudaDeviceReset discards the array with the device's context and
 *   leaves the cached address stale: do not call this entry point after resetting the device.
 * Failure: as for lls_lowp_projection, a device wait that gives up leaves R12 and R12l as NaN
 *   (f = 0); the error word itself is inside the library's array and is not visible.
 * Sharing: all calls in the process use the same array, which keeps the last call's
 *   contents; each call clears the error word itself on the given stream. Calls whose work
 *   overlaps on the GPU (different streams without ordering, several host threads) race on
 *   the array and give wrong results: order them on one stream or with events.
 * Errors: LLS_ERR_ARG, LLS_ERR_TOO_LARGE, LLS_ERR_UNSUPPORTED (alignment, device index >= 64),
 *   LLS_ERR_CUDA.
 * -------------------------------------------------------------------------- */
#define LLS_NOALLOC_SCRATCH_BYTES ((size_t)4 << 20)
int lls_lowp_projection_noalloc(int m, int w1, int w2, int prec, const void* Q1l, const void* A2l,
                                int ldh, const int* e, float* R12, int ldr, void* R12l, int ldrl,
                                int* f, cudaStream_t stream);

#ifdef __cplusplus
}
#endif
#endif /* LLS_GB300_H */
