// Internal launch interfaces between the library's translation units.
#pragma once
#include "common.cuh"

namespace lls {

constexpr int kMaxPanelLevels = 8;

// Implementation choices that leave the arithmetic of the method unchanged (the same rounding
// points, the same fixed summation orders within each kernel); the autotuner picks them per
// shape. The environment switches LLS_NODE and LLS_GEMM set the defaults, for comparisons.
struct Knobs {
    int node_mode = 0;      // 0: the lowest nodes with their two panels, and the narrow nodes, as
                            //    single launches; 1: narrow nodes as single launches, the lowest
                            //    nodes' panels separate; 2: every node as four launches
    int gemm_kernel = 0;    // products of the wide nodes: 0 persistent, 1 one output tile per CTA,
                            // 2 persistent update with the one-tile-per-CTA projection
    int batched_ctas = 0;   // batched solver: CTAs per SM, 0 = as many as fit
    int krylov_ctas = 0;    // CTAs of the Krylov kernel, 0 = from the problem size
};
Knobs default_knobs();

// ---- panel (panel.cu) -------------------------------------------------------------------
struct PanelCall {
    float* W; int ldw;
    void* Wh; int ldh;
    float* R; int ldr;
    int m, c0, b;
    int lowp;              // 0 FP16, 1 BF16, 3 none
    float* rbuf; float* qbuf; unsigned* cnt;
    int* err;
    int leaf = 0;          // 0 CGS2, 1 MGS (Alg. 4; one-level panels only)
};
// cnt[kFlatBarWord .. +kFlatBarWords): the grid barrier (count, generation) of the one-level
// panel, apart from the multi-level panel's words so that the two can follow one another
constexpr int kFlatBarWord = 2, kFlatBarWords = 2;
void panel_scratch_sizes(int m, size_t& rbuf_floats, size_t& qbuf_floats, size_t& cnt_words);
int panel_qr(const PanelCall& c, cudaStream_t st);
// One-level-tree variant (panel_flat.cu); LLS_ERR_UNSUPPORTED when the panel needs a deeper tree.
int panel_flat_qr(const PanelCall& c, cudaStream_t st);
// Debug build: arms a planted fault of the CAQR panel kernels (1: out-of-range Q stores, 2: a
// grid barrier that cannot complete) or disarms it (0).
int panel_debug_inject(int mode);
// Two one-level panels and the recursion node between them in one cooperative launch
// (panel_flat.cu): columns [c0, c0 + w1) and [c0 + w1, c0 + w1 + w2), 8 < w1 <= 16,
// 1 <= w2 <= w1, FP16 or BF16 products. LLS_ERR_UNSUPPORTED (nothing launched) otherwise.
struct BlockCall {
    float* W; int ldw;
    void* Wh; int ldh;
    float* R; int ldr;
    int m, c0, w1, w2;
    int lowp;              // 0 FP16, 1 BF16
    float* rbuf; unsigned* cnt;
    float* part; size_t part_floats;
    int* err;
};
int block_fused_qr(const BlockCall& c, cudaStream_t st);
bool block_fused_supported(const BlockCall& c);   // the shape checks of block_fused_qr alone
size_t block_fused_part_floats();                  // partial sums the block needs at most

// ---- scale / cast (cast.cu) ---------------------------------------------------------------
// For columns [c0, c0 + w) of the FP32 matrix X (m rows, ldx): e_j = column scale exponent
// (FP16 rule; 0 for BF16), Xh[:, j] = round(X[:, j] * 2^e_j). Writes exps[j - c0].
int scale_cast_columns(const float* X, int ldx, int m, int c0, int w, void* Xh, int ldh,
                       int lowp, int* exps, cudaStream_t st);
// row-major copy of columns [c0, c0 + w) of a column-major 8-bit matrix (lowp 2 only)
int rowmajor_copy8(const void* X, int ldx, int m, int c0, int w, void* T, int ldt, cudaStream_t st);

// ---- tensor-core products (gemm_tc.cu) ----------------------------------------------------
// G1 (Alg. 2, projection): part[s] = Q1l^T A2l over K-split s; then R12 = sum_s part[s] * 2^-e_j
//     written to R (FP32), and R12l = round(R12 * 2^f_j) with its own column exponents f_j.
// G2 (Alg. 2, update): A2 -= (Q1l R12l) * 2^-f_j, FP32 in place.
struct ProjCall {
    const void* Q1l; const void* A2l; int ldh;   // low-precision operands (column-major, ld ldh)
    int m, w1, w2;                                // M = w1, N = w2, K = m
    const int* e;                                 // A2 column exponents (w2)
    const int* sq = nullptr;                      // FP8: Q1 column exponents (w1), else null
    float* R12; int ldr;                          // FP32 output block of R
    void* R12l; int ldrl;                         // low-precision scaled copy for G2 (w1 x w2)
    int* f;                                       // R12 column exponents (w2)
    float* part; size_t part_floats;              // split-K partials scratch
    int lowp;
    int* err;                                     // device error word (bounded waits)
    int gemm_kernel = 0;                          // Knobs::gemm_kernel
};
struct UpdCall {
    const void* Q1l; int ldh;                     // m x w1 low precision (M-major A operand)
    const void* QT = nullptr; int ldq = 0;        // FP8: Q1 row-major (K-major A operand), ldq bytes
    const void* R12l; int ldrl;                   // w1 x w2 low precision (scaled by 2^f)
    const int* f;
    float* A2; int ldw;                           // m x w2 FP32, updated in place
    int m, w1, w2;
    int lowp;
    int* err;
    int gemm_kernel = 0;                          // Knobs::gemm_kernel
};
size_t proj_partial_floats(int m, int w1, int w2);
// Narrow node (w1 <= 32, FP16/BF16) as one cooperative launch (node_fused.cu): the same
// products as gemm_projection + gemm_update without the separate cast and reduce passes.
// LLS_ERR_UNSUPPORTED (nothing launched) when the node does not qualify.
struct NodeCall {
    float* W; int ldw;                            // FP32 work matrix (Q1 and A2 columns)
    const void* Wh; int ldh;                      // product-precision copy holding Q1l
    int m, c0, w1, w2, lowp;
    float* R; int ldr;
    float* part; size_t part_floats;              // >= node_fused_part_floats(m)
    void* R12l; int* f;                           // >= 32 x 32 low-precision values; w2 ints
    unsigned* bar;                                // 2 words, zero on entry (left zero)
    int* err;
};
size_t node_fused_part_floats(int m);
int node_fused(const NodeCall& c, cudaStream_t st);
int gemm_projection(const ProjCall& c, cudaStream_t st);
int gemm_update(const UpdCall& c, cudaStream_t st);

// ---- FP32 SIMT GEMM (gemm_simt.cu): reference-precision products and the R^-1 recursion --
// C = alpha * op(A) op(B) + beta * C, column-major, op(X) = X or X^T.
int sgemm(bool ta, bool tb, int M, int N, int K, float alpha, const float* A, int lda,
          const float* B, int ldb, float beta, float* C, int ldc, cudaStream_t st);

// ---- triangular inverse (trinv.cu) ----------------------------------------------------------
// Minv = R^{-1} (upper triangular, n x n, ld n) via diagonal-block inverses and the recursion
// M12 = -M11 R12 M22 over the same column split as the QR; Mt = Minv^T. tmp: n*n floats.
// C = U V for upper-triangular n x n U, V (column-major); C (distinct from U and V) is
// upper triangular with zeros written below the diagonal. FP32.
int triu_product(const float* U, int ldu, const float* V, int ldv, float* C, int ldc, int n, cudaStream_t st);
int tri_inverse(const float* R, int ldr, int n, int pw, float* Minv, float* Mt, float* tmp,
                int* dev_err, cudaStream_t st);

// ---- Krylov (krylov.cu) -----------------------------------------------------------------------
struct KrylovCall {
    int m, n;
    const float* A; int lda;
    const double* b;
    double* x;
    const float* Minv;      // R^{-1}, column-major n x n
    const float* Mt;        // (R^{-1})^T, column-major n x n
    int method;             // lls_krylov
    int target;             // lls_target
    double tol;
    int max_iter;
    void* scratch; size_t scratch_bytes;
    int* dev_err;
    double* dev_info;       // [iters, eta, fwd, res, atr, anorm, xnorm, status]
    int x_zero = 1;         // 1: start from x = 0; 0: start from the x the vector holds
    double* hist = nullptr; // kHistLen doubles: the stop quantity after each iteration, or null
    unsigned long long* phases = nullptr;   // kPhaseLen entries: CGLS phase log (LLS_LOG=2), or null
    int ctas = 0;           // CTAs of the persistent kernel, 0 = from the problem size
};
// CTAs the Krylov kernel takes for an m x n problem when not told otherwise.
int krylov_default_ctas(int m, int n);
constexpr int kHistLen = 4096;   // iterations whose stop quantity the history keeps
constexpr int kPhaseLen = 4096;  // entries of the CGLS phase log
// one_pass: room for the one-pass CGLS engine's row-block copy of A (used when n <= 4096).
size_t krylov_scratch_bytes(int m, int n, int grid, bool one_pass = false);
int krylov_solve(const KrylovCall& c, cudaStream_t st);

// Adjoint (krylov.cu): z = (A^T A)^{-1} g by M M^T-preconditioned CG, then
// gb = A z and gA = (b - A x) z^T - (A z) x^T.
struct AdjointCall {
    int m, n;
    const float* A; int lda;
    const double* b; const double* x; const double* g;
    const float* Minv; const float* Mt;
    double* z;              // n, output
    float* gA; int ldga;    // m x n FP32 output
    double* gb;             // m FP64 output
    double tol; int max_iter;
    void* scratch; size_t scratch_bytes;
    int* dev_err; double* dev_info;
};
int adjoint_solve(const AdjointCall& c, cudaStream_t st);

// ---- batched solver (batched.cu) -----------------------------------------------------------
bool batched_supported(int m, int n);
size_t batched_workspace_bytes(int batch, const int* m, const int* n);
double* batched_info_ptr(void* ws, int batch, const int* m, const int* n);
int batched_upload(int batch, const int* m, const int* n, const float* const* A, const int* lda,
                   const double* const* b, double* const* x, float* const* Rout, const int* ldr,
                   void* ws, size_t ws_bytes, cudaStream_t st);
int batched_execute(int batch, const int* m, const int* n, void* ws, const lls_options& o, int ctas_per_sm,
                    cudaStream_t st);
// The adjoint of a batch of solves in one persistent launch (each CTA whole problems).
size_t batched_adjoint_workspace_bytes(int batch, const int* m, const int* n);
int batched_adjoint(int batch, const int* m, const int* n, const float* const* A, const int* lda,
                    const double* const* b, const double* const* x, const float* const* R, const int* ldr,
                    const double* const* grad_x, float* const* grad_A, const int* ldga, double* const* grad_b,
                    void* ws, size_t ws_bytes, double tol, int max_iter, cudaStream_t st);

// ---- graph replay (graph.cu) -----------------------------------------------------------------
// Identity of one call: plain-old-data, compared bytewise (zero-initialize before filling).
struct GraphKey {
    int op, device;
    int ints[8];
    const void* ptrs[8];
    size_t ws_bytes;
    lls_options opts;
    Knobs knobs;
};
// Enqueues one call on `st`; ev (may be null) receives 3 phase events; `capturing` selects
// external event-record nodes.
typedef int (*EnqueueFn)(void* ctx, cudaStream_t st, cudaEvent_t* ev, bool capturing);
int run_graphed(const GraphKey& key, cudaStream_t st, EnqueueFn fn, void* ctx, cudaEvent_t* ev_out);
void record_phase(cudaEvent_t ev, cudaStream_t st, bool capturing);

// ---- direct solve with the mixed-precision factors (direct.cu) ------------------------------
// x = M (Q^T b) with M = R^{-1} given as Mt = M^T (column-major n x n, ld n); Q m x n FP32.
size_t direct_start_scratch_bytes(int m, int n);
int direct_start(const float* Q, int ldq, int m, int n, const double* b, const float* Mt, double* x, void* scratch,
                 size_t scratch_bytes, cudaStream_t st);

// ---- misc (util.cu) -------------------------------------------------------------------------
int copy_matrix(const float* src, int lds, float* dst, int ldd, int m, int n, cudaStream_t st);
int check_diag(const float* R, int ldr, int n, int* dev_err, cudaStream_t st);
int poison_diag_on_error(float* R, int ldr, int n, const int* dev_err, cudaStream_t st);
int zero_lower(float* R, int ldr, int n, cudaStream_t st);

}  // namespace lls
