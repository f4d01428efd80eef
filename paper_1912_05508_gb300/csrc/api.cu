// C ABI: qr_factor and lls_solve (see include/lls_gb300.h), and the recursion driver.
//
// qr_factor runs Alg. 2 (recursive Gram-Schmidt QR, Eq. recqr) depth first on the host,
// enqueueing for every internal node of width w = w1 + w2:
//   scale/cast of A2 (columns [c0+w1, c0+w))          -> low-precision A2 and exponents e
//   projection R12 = Q1^T A2 (Alg. 2 line 8)          -> FP32 R12 block of R, scaled low-precision R12
//   update A2 <- A2 - Q1 R12 (Alg. 2 line 9)          -> FP32 in place
// and for every leaf (<= panel_width columns) the CAQR panel (Eq. caqr). All of it is
// asynchronous on the caller's stream; nothing is allocated.
#include <string.h>

#include "common.cuh"
#include "kernels.cuh"

namespace lls {

int fro_sumsq(const float* A, int lda, int m, int n, double* part, double* out, cudaStream_t st);
int simt_projection_f32(const float* Q1, const float* A2, int ldw, int m, int w1, int w2,
                        float* R12, int ldr, float* part, cudaStream_t st);
int simt_update_f32(const float* Q1, int ldw, const float* R12, int ldr, float* A2, int m, int w1,
                    int w2, cudaStream_t st);
size_t simt_partial_floats(int m, int w1, int w2);

static int split_point(int w, int pw) { return pw * ceil_div(w, 2 * pw); }

static void resolve(const lls_options* o, lls_options& r) {
    lls_default_options(&r);
    if (!o) return;
    r = *o;
    if (r.panel_width <= 0) r.panel_width = 32;
    if (r.leaf_rows <= 0) r.leaf_rows = 256;
    if (r.max_iter <= 0) r.max_iter = 200;
    if (r.tol <= 0.0) r.tol = r.target == LLS_TARGET_FP32 ? 1e-6 : 1e-12;
}

static bool valid_opts(const lls_options& o) {
    if (o.gemm_prec != LLS_PREC_FP16 && o.gemm_prec != LLS_PREC_BF16 && o.gemm_prec != LLS_PREC_FP32) return false;
    if (o.target != LLS_TARGET_FP32 && o.target != LLS_TARGET_FP64) return false;
    if (o.krylov != LLS_KRYLOV_CGLS && o.krylov != LLS_KRYLOV_LSQR) return false;
    if (o.panel_width < 1 || o.panel_width > 32) return false;
    if (o.leaf_rows != 256) return false;
    return true;
}

// Largest split-K partial buffer over all internal nodes of the recursion.
static size_t max_partial(int m, int c0, int w, int pw, bool lowp) {
    if (w <= pw) return 0;
    int w1 = split_point(w, pw), w2 = w - w1;
    size_t here = lowp ? proj_partial_floats(m, w1, w2) : simt_partial_floats(m, w1, w2);
    size_t l = max_partial(m, c0, w1, pw, lowp), r = max_partial(m, c0 + w1, w2, pw, lowp);
    size_t mx = here > l ? here : l;
    return mx > r ? mx : r;
}

struct QrWs {
    float* W; int ldw;
    void* Wh; int ldh;
    float* part; size_t part_floats;
    void* R12l; int* eA; int* f;
    float* rbuf; float* qbuf; unsigned* cnt; size_t cnt_words;
    int* err;
    double* dinfo;     // 16 doubles of device-side results
    double* red;       // 8192 doubles of reduction partials
};

static int lowp_code(int prec) { return prec == LLS_PREC_FP16 ? 0 : (prec == LLS_PREC_BF16 ? 1 : 3); }

static void qr_layout(WsArena& ar, int m, int n, const lls_options& o, QrWs& w) {
    const bool lowp = o.gemm_prec != LLS_PREC_FP32;
    w.ldw = (int)align_up((size_t)m, 64);
    w.ldh = w.ldw;
    w.W = ar.take<float>((size_t)w.ldw * n);
    w.Wh = lowp ? (void*)ar.take<uint16_t>((size_t)w.ldh * n) : nullptr;
    w.part_floats = max_partial(m, 0, n, o.panel_width, lowp);
    if (w.part_floats == 0) w.part_floats = 1;
    w.part = ar.take<float>(w.part_floats);
    size_t r12 = (size_t)(n / 2 + 32) * (size_t)(n / 2 + 32);
    w.R12l = lowp ? (void*)ar.take<uint16_t>(r12) : nullptr;
    w.eA = ar.take<int>(n);
    w.f = ar.take<int>(n);
    size_t rb, qb, cw;
    panel_scratch_sizes(m, rb, qb, cw);
    w.rbuf = ar.take<float>(rb);
    w.qbuf = ar.take<float>(qb);
    w.cnt = ar.take<unsigned>(cw);
    w.cnt_words = cw;
    w.err = ar.take<int>(16);
    w.dinfo = ar.take<double>(16);
    w.red = ar.take<double>(8192);
}

struct QrCtx {
    int m, n, pw, lowp;
    QrWs w;
    float* R; int ldr;
    cudaStream_t st;
};

static int qr_rec(QrCtx& c, int c0, int w) {
    if (w <= c.pw) {
        PanelCall p;
        p.W = c.w.W; p.ldw = c.w.ldw; p.Wh = c.w.Wh; p.ldh = c.w.ldh; p.R = c.R; p.ldr = c.ldr;
        p.m = c.m; p.c0 = c0; p.b = w; p.lowp = c.lowp;
        p.rbuf = c.w.rbuf; p.qbuf = c.w.qbuf; p.cnt = c.w.cnt;
        return panel_qr(p, c.st);
    }
    const int w1 = split_point(w, c.pw), w2 = w - w1;
    LLS_TRY(qr_rec(c, c0, w1));
    float* R12 = c.R + (size_t)c0 + (size_t)(c0 + w1) * c.ldr;
    float* A2 = c.w.W + (size_t)(c0 + w1) * c.w.ldw;
    const float* Q1 = c.w.W + (size_t)c0 * c.w.ldw;
    if (c.lowp == 3) {
        LLS_TRY(simt_projection_f32(Q1, A2, c.w.ldw, c.m, w1, w2, R12, c.ldr, c.w.part, c.st));
        LLS_TRY(simt_update_f32(Q1, c.w.ldw, R12, c.ldr, A2, c.m, w1, w2, c.st));
    } else {
        const size_t esz = 2;
        const char* Whb = (const char*)c.w.Wh;
        LLS_TRY(scale_cast_columns(c.w.W, c.w.ldw, c.m, c0 + w1, w2, c.w.Wh, c.w.ldh, c.lowp, c.w.eA, c.st));
        ProjCall pc;
        pc.Q1l = Whb + esz * (size_t)c0 * c.w.ldh;
        pc.A2l = Whb + esz * (size_t)(c0 + w1) * c.w.ldh;
        pc.ldh = c.w.ldh; pc.m = c.m; pc.w1 = w1; pc.w2 = w2; pc.e = c.w.eA;
        pc.R12 = R12; pc.ldr = c.ldr; pc.R12l = c.w.R12l; pc.ldrl = w1; pc.f = c.w.f;
        pc.part = c.w.part; pc.part_floats = c.w.part_floats; pc.lowp = c.lowp;
        LLS_TRY(gemm_projection(pc, c.st));
        UpdCall uc;
        uc.Q1l = pc.Q1l; uc.ldh = c.w.ldh; uc.R12l = c.w.R12l; uc.ldrl = w1; uc.f = c.w.f;
        uc.A2 = A2; uc.ldw = c.w.ldw; uc.m = c.m; uc.w1 = w1; uc.w2 = w2; uc.lowp = c.lowp;
        LLS_TRY(gemm_update(uc, c.st));
    }
    return qr_rec(c, c0 + w1, w2);
}

static int run_qr(int m, int n, const float* A, int lda, float* R, int ldr, const lls_options& o,
                  QrWs& w, cudaStream_t st) {
    LLS_CUDA_TRY(cudaMemsetAsync(w.cnt, 0, sizeof(unsigned) * w.cnt_words, st));
    LLS_TRY(copy_matrix(A, lda, w.W, w.ldw, m, n, st));
    LLS_CUDA_TRY(cudaMemset2DAsync(R, sizeof(float) * (size_t)ldr, 0, sizeof(float) * (size_t)n, (size_t)n, st));
    QrCtx c;
    c.m = m; c.n = n; c.pw = o.panel_width; c.lowp = lowp_code(o.gemm_prec);
    c.w = w; c.R = R; c.ldr = ldr; c.st = st;
    return qr_rec(c, 0, n);
}

}  // namespace lls

#include <atomic>

namespace lls {
static std::atomic<unsigned long long> g_launches{0};
void note_launch() { g_launches.fetch_add(1, std::memory_order_relaxed); }
}  // namespace lls

using namespace lls;

extern "C" {

unsigned long long lls_kernel_launch_count(void) { return g_launches.load(std::memory_order_relaxed); }

void lls_default_options(lls_options* o) {
    if (!o) return;
    memset(o, 0, sizeof(*o));
    o->gemm_prec = LLS_PREC_FP16;
    o->target = LLS_TARGET_FP64;
    o->tol = 0.0;
    o->max_iter = 200;
    o->panel_width = 32;
    o->krylov = LLS_KRYLOV_CGLS;
    o->leaf_rows = 256;
}

const char* lls_status_string(int s) {
    switch (s) {
        case LLS_OK: return "ok";
        case LLS_NOT_CONVERGED: return "not converged (iteration limit)";
        case LLS_ERR_ARG: return "invalid argument";
        case LLS_ERR_SINGULAR: return "singular or non-finite R";
        case LLS_ERR_CUDA: return "CUDA error";
        case LLS_ERR_WORKSPACE: return "workspace too small or misaligned";
        case LLS_ERR_TIMEOUT: return "device wait timed out";
        case LLS_ERR_UNSUPPORTED: return "unsupported option combination";
        default: return "unknown status";
    }
}

size_t qr_factor_workspace_size(int m, int n, const lls_options* opts) {
    lls_options o;
    resolve(opts, o);
    if (n < 1 || m < n || !valid_opts(o)) return 0;
    WsArena ar(nullptr, SIZE_MAX);
    QrWs w;
    qr_layout(ar, m, n, o, w);
    return ar.off;
}

int qr_factor(int m, int n, const float* A, int lda, float* Q, int ldq, float* R, int ldr,
              void* ws, size_t ws_bytes, const lls_options* opts, cudaStream_t stream) {
    lls_options o;
    resolve(opts, o);
    if (n < 1 || m < n || lda < m || ldr < n || !A || !R || !ws) return LLS_ERR_ARG;
    if (Q && ldq < m) return LLS_ERR_ARG;
    if (!valid_opts(o)) return LLS_ERR_ARG;
    if (((uintptr_t)ws & 255) != 0) return LLS_ERR_WORKSPACE;
    WsArena ar(ws, ws_bytes);
    QrWs w;
    qr_layout(ar, m, n, o, w);
    if (!ar.ok) return LLS_ERR_WORKSPACE;
    LLS_TRY(run_qr(m, n, A, lda, R, ldr, o, w, stream));
    if (Q) LLS_TRY(copy_matrix(w.W, w.ldw, Q, ldq, m, n, stream));
    return LLS_OK;
}

static void lls_layout(WsArena& ar, int m, int n, const lls_options& o, QrWs& w, float*& R,
                       float*& Minv, float*& Mt, float*& tmp, void*& ks, size_t& ks_bytes) {
    qr_layout(ar, m, n, o, w);
    R = ar.take<float>((size_t)n * n);
    Minv = ar.take<float>((size_t)n * n);
    Mt = ar.take<float>((size_t)n * n);
    tmp = ar.take<float>((size_t)n * n);
    ks_bytes = krylov_scratch_bytes(m, n, 0);
    ks = ar.take<char>(ks_bytes);
}

size_t lls_solve_workspace_size(int m, int n, const lls_options* opts) {
    lls_options o;
    resolve(opts, o);
    if (n < 1 || m < n || !valid_opts(o)) return 0;
    WsArena ar(nullptr, SIZE_MAX);
    QrWs w; float *R, *Mi, *Mt, *tmp; void* ks; size_t kb;
    lls_layout(ar, m, n, o, w, R, Mi, Mt, tmp, ks, kb);
    return ar.off;
}

int lls_solve(int m, int n, const float* A, int lda, const double* b, double* x, float* R_out,
              int ldr, void* ws, size_t ws_bytes, const lls_options* opts, lls_info* info,
              cudaStream_t stream) {
    lls_options o;
    resolve(opts, o);
    if (info) memset(info, 0, sizeof(*info));
    if (n < 1 || m < n || lda < m || !A || !b || !x || !ws) return LLS_ERR_ARG;
    if (R_out && ldr < n) return LLS_ERR_ARG;
    if (!valid_opts(o)) return LLS_ERR_ARG;
    if (o.krylov != LLS_KRYLOV_CGLS) return LLS_ERR_UNSUPPORTED;
    if (((uintptr_t)ws & 255) != 0) return LLS_ERR_WORKSPACE;
    WsArena ar(ws, ws_bytes);
    QrWs w; float *R, *Minv, *Mt, *tmp; void* ks; size_t kb;
    lls_layout(ar, m, n, o, w, R, Minv, Mt, tmp, ks, kb);
    if (!ar.ok) return LLS_ERR_WORKSPACE;

    cudaEvent_t ev[3] = {nullptr, nullptr, nullptr};
    if (info)
        for (auto& e : ev) LLS_CUDA_TRY(cudaEventCreate(&e));
    if (info) LLS_CUDA_TRY(cudaEventRecord(ev[0], stream));
    LLS_CUDA_TRY(cudaMemsetAsync(w.err, 0, sizeof(int) * 16, stream));
    LLS_CUDA_TRY(cudaMemsetAsync(w.dinfo, 0, sizeof(double) * 16, stream));
    LLS_TRY(run_qr(m, n, A, lda, R, n, o, w, stream));
    if (R_out) LLS_TRY(copy_matrix(R, n, R_out, ldr, n, n, stream));
    LLS_TRY(check_diag(R, n, n, w.err, stream));
    LLS_TRY(tri_inverse(R, n, n, o.panel_width, Minv, Mt, tmp, w.err, stream));
    LLS_TRY(fro_sumsq(A, lda, m, n, w.red, w.dinfo + 8, stream));
    LLS_TRY(fro_sumsq(Minv, n, n, n, w.red + 4096, w.dinfo + 9, stream));
    if (info) LLS_CUDA_TRY(cudaEventRecord(ev[1], stream));
    KrylovCall kc;
    kc.m = m; kc.n = n; kc.A = A; kc.lda = lda; kc.b = b; kc.x = x; kc.Minv = Minv; kc.Mt = Mt;
    kc.method = o.krylov; kc.target = o.target; kc.tol = o.tol; kc.max_iter = o.max_iter;
    kc.scratch = ks; kc.scratch_bytes = kb; kc.dev_err = w.err; kc.dev_info = w.dinfo;
    LLS_TRY(krylov_solve(kc, stream));
    if (!info) return LLS_OK;
    LLS_CUDA_TRY(cudaEventRecord(ev[2], stream));
    double hinfo[16];
    int herr = 0;
    LLS_CUDA_TRY(cudaMemcpyAsync(hinfo, w.dinfo, sizeof(hinfo), cudaMemcpyDeviceToHost, stream));
    LLS_CUDA_TRY(cudaMemcpyAsync(&herr, w.err, sizeof(int), cudaMemcpyDeviceToHost, stream));
    LLS_CUDA_TRY(cudaStreamSynchronize(stream));
    cudaEventElapsedTime(&info->qr_ms, ev[0], ev[1]);
    cudaEventElapsedTime(&info->krylov_ms, ev[1], ev[2]);
    for (auto& e : ev) cudaEventDestroy(e);
    info->iters = (int)hinfo[0];
    info->eta = hinfo[1];
    info->fwd_est = hinfo[2];
    info->res_norm = hinfo[3];
    info->atr_norm = hinfo[4];
    info->anorm_f = hinfo[5];
    info->xnorm = hinfo[6];
    info->a_passes = (int)hinfo[10];
    info->m_passes = (int)hinfo[11];
    int st = (int)hinfo[7] == 0 ? LLS_OK : LLS_NOT_CONVERGED;
    if (herr == DEV_SINGULAR) st = LLS_ERR_SINGULAR;
    else if (herr == DEV_TIMEOUT) st = LLS_ERR_TIMEOUT;
    else if (herr != DEV_OK) st = LLS_ERR_CUDA;
    info->status = st;
    return st;
}

}  // extern "C"
