// C ABI: qr_factor and lls_solve (see include/lls_gb300.h), and the recursion driver.
//
// qr_factor runs Alg. 2 (recursive Gram-Schmidt QR, Eq. recqr) depth first on the host,
// enqueueing for every internal node of width w = w1 + w2:
//   scale/cast of A2 (columns [c0+w1, c0+w))          -> low-precision A2 and exponents e
//   projection R12 = Q1^T A2 (Alg. 2)                 -> FP32 R12 block of R, scaled low-precision R12
//   update A2 <- A2 - Q1 R12 (Alg. 2)                 -> FP32 in place
// and for every leaf (<= panel_width columns) the CAQR panel (Eq. caqr). All of it is
// asynchronous on the caller's stream; nothing is allocated.
#include <stdio.h>
#include <stdlib.h>

#include <mutex>
#include <string.h>

#include <map>
#include <algorithm>
#include <vector>

#include "common.cuh"
#include "kernels.cuh"

namespace lls {

int fro_sumsq(const float* A, int lda, int m, int n, double* part, double* out, cudaStream_t st);
int copy_fro_sumsq(const float* A, int lda, float* W, int ldw, int m, int n, double* part, double* out,
                   cudaStream_t st);
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
    if (r.panel_width <= 0) r.panel_width = 16;
    if (r.leaf_rows <= 0) r.leaf_rows = 256;
    if (r.max_iter <= 0) r.max_iter = 200;
    if (r.tol <= 0.0) r.tol = r.target == LLS_TARGET_FP32 ? 1e-6 : 1e-12;
}

static bool valid_opts(const lls_options& o) {
    if (o.gemm_prec != LLS_PREC_FP16 && o.gemm_prec != LLS_PREC_BF16 && o.gemm_prec != LLS_PREC_FP8 &&
        o.gemm_prec != LLS_PREC_FP32)
        return false;
    if (o.target != LLS_TARGET_FP32 && o.target != LLS_TARGET_FP64) return false;
    if (o.krylov != LLS_KRYLOV_CGLS && o.krylov != LLS_KRYLOV_LSQR) return false;
    if (o.panel_width < 1 || o.panel_width > 32) return false;
    if (o.gemm_prec == LLS_PREC_FP8 && o.panel_width % 16 != 0) return false;   // 16-byte aligned FP8 slices
    if (o.leaf_rows != 256) return false;
    if (o.reorth != 0 && o.reorth != 1) return false;
    if (o.panel_leaf != 0 && o.panel_leaf != 1) return false;
    if (o.x0 < LLS_X0_ZERO || o.x0 > LLS_X0_DIRECT) return false;
    return true;
}

// ---- tuned settings: recorded by lls_autotune / lls_tuning_set, used when the caller leaves
// panel_width at 0 ("auto") -----------------------------------------------------------------
struct TuneKey {
    int v[9];
    bool operator<(const TuneKey& o) const { return memcmp(v, o.v, sizeof(v)) < 0; }
};
static std::mutex g_tune_mu;
static std::map<TuneKey, lls_tuning> g_tune;

static TuneKey tune_key(int kind, int m, int n, const lls_options& o) {
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) {
        cudaGetLastError();
        dev = 0;
    }
    TuneKey k;
    const int v[9] = {dev, kind, m, n, o.gemm_prec, o.target, o.krylov, o.reorth, o.panel_leaf};
    memcpy(k.v, v, sizeof(v));
    return k;
}

static bool tuned_lookup(int kind, int m, int n, const lls_options& o, lls_tuning& t) {
    std::lock_guard<std::mutex> lk(g_tune_mu);
    auto it = g_tune.find(tune_key(kind, m, n, o));
    if (it == g_tune.end()) return false;
    t = it->second;
    return true;
}

static bool auto_width(const lls_options* opts) { return !opts || opts->panel_width <= 0; }

// Options and implementation choices of a call: the caller's options with defaults filled in;
// with panel_width 0, the settings recorded for this shape if there are any.
static void resolve_settings(const lls_options* opts, int kind, int m, int n, lls_options& o, Knobs& k) {
    resolve(opts, o);
    k = default_knobs();
    if (!auto_width(opts)) return;
    lls_tuning t;
    if (!tuned_lookup(kind, m, n, o, t)) return;
    if (kind == 0 && t.panel_width >= 1 && t.panel_width <= 32) {
        lls_options c = o;
        c.panel_width = t.panel_width;
        if (valid_opts(c)) o.panel_width = t.panel_width;
    }
    if (t.node_mode >= 0 && t.node_mode <= 2) k.node_mode = t.node_mode;
    if (t.gemm_kernel >= 0 && t.gemm_kernel <= 2) k.gemm_kernel = t.gemm_kernel;
    if (t.batched_ctas_per_sm >= 0) k.batched_ctas = t.batched_ctas_per_sm;
    if (t.krylov_ctas >= 0) k.krylov_ctas = t.krylov_ctas;
}

// Panel widths an "auto" call may end up with; its workspace is sized for the largest need.
static const int kTuneWidths[3] = {8, 16, 32};

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
    uint8_t* QT; int ldq; int* sQ;   // FP8 only: row-major copy of Q and its column exponents
    float* R1; float* Rt;            // re-orthogonalization: the first pass's R, and R2 R1 (n x n)
    float* rbuf; float* qbuf; unsigned* cnt; size_t cnt_words;
    unsigned* nbar;                  // fused narrow nodes: grid barrier (2)
    int* err;
    double* dinfo;     // 16 doubles of device-side results
    double* red;       // 8192 doubles of reduction partials
};

static int lowp_code(int prec) {
    return prec == LLS_PREC_FP16 ? 0 : (prec == LLS_PREC_BF16 ? 1 : (prec == LLS_PREC_FP8 ? 2 : 3));
}

static void qr_layout(WsArena& ar, int m, int n, const lls_options& o, QrWs& w) {
    const bool lowp = o.gemm_prec != LLS_PREC_FP32;
    w.ldw = (int)align_up((size_t)m, 64);
    w.ldh = w.ldw;
    w.W = ar.take<float>((size_t)w.ldw * n);
    w.Wh = lowp ? (void*)ar.take<uint16_t>((size_t)w.ldh * n) : nullptr;
    w.part_floats = max_partial(m, 0, n, o.panel_width, lowp);
    if (o.gemm_prec == LLS_PREC_FP16 || o.gemm_prec == LLS_PREC_BF16) {
        const size_t nf = node_fused_part_floats(m);
        if (nf > w.part_floats) w.part_floats = nf;
    }
    if (w.part_floats == 0) w.part_floats = 1;
    w.part = ar.take<float>(w.part_floats);
    size_t r12 = (size_t)(n / 2 + 32) * (size_t)(n / 2 + 32);
    w.R12l = lowp ? (void*)ar.take<uint16_t>(r12) : nullptr;
    w.eA = ar.take<int>(n);
    w.f = ar.take<int>(n);
    const bool f8 = o.gemm_prec == LLS_PREC_FP8;
    w.ldq = (int)align_up((size_t)n, 16);
    w.QT = f8 ? ar.take<uint8_t>((size_t)m * w.ldq) : nullptr;
    w.sQ = f8 ? ar.take<int>(n) : nullptr;
    w.R1 = o.reorth ? ar.take<float>((size_t)n * n) : nullptr;
    w.Rt = o.reorth ? ar.take<float>((size_t)n * n) : nullptr;
    size_t rb, qb, cw;
    panel_scratch_sizes(m, rb, qb, cw);
    w.rbuf = ar.take<float>(rb);
    w.qbuf = ar.take<float>(qb);
    w.cnt = ar.take<unsigned>(cw);
    w.cnt_words = cw;
    w.nbar = ar.take<unsigned>(4);      // the grid barrier's 64-bit word, 8-byte aligned
    w.err = ar.take<int>(16);
    w.dinfo = ar.take<double>(16);
    w.red = ar.take<double>(8192);
}

// Columns of W that arrive in chunks on another stream (the host-input solve): chunk k covers
// columns [start[k], start[k + 1]) and is complete when ev[k] fires. The recursion first
// touches columns in increasing order, so it waits for the chunks up to the last column a
// launch touches, just before that launch.
constexpr int kMaxChunks = 32;
struct ColumnGate {
    int count = 0;
    int start[kMaxChunks + 1];
    cudaEvent_t ev[kMaxChunks];
    int ready = 0;                      // chunks the stream already waits for
};

struct QrCtx {
    int m, n, pw, lowp, leaf;
    Knobs k;
    QrWs w;
    float* R; int ldr;
    cudaStream_t st;
    ColumnGate* gate = nullptr;
};

static int gate_upto(QrCtx& c, int col_end) {
    if (!c.gate) return LLS_OK;
    ColumnGate& g = *c.gate;
    while (g.ready < g.count && g.start[g.ready] < col_end) {
        LLS_CUDA_TRY(cudaStreamWaitEvent(c.st, g.ev[g.ready], 0));
        ++g.ready;
    }
    return LLS_OK;
}

// The defaults of the implementation choices (Knobs). LLS_NODE=split keeps every node on the
// four-kernel path, LLS_NODE=node runs narrow nodes as one launch each but keeps the lowest
// nodes' panels separate, LLS_GEMM=cta runs the wide nodes' products one output tile per CTA
// (all for comparisons).
Knobs default_knobs() {
    static const Knobs k = [] {
        Knobs d;
        const char* v = getenv("LLS_NODE");
        if (v && v[0] == 's') d.node_mode = 2;
        else if (v && v[0] == 'n') d.node_mode = 1;
        const char* g = getenv("LLS_GEMM");
        if (g && g[0] == 'c') d.gemm_kernel = 1;
        return d;
    }();
    return k;
}

static int qr_rec(QrCtx& c, int c0, int w) {
    if (w <= c.pw) {
        LLS_TRY(gate_upto(c, c0 + w));
        PanelCall p;
        p.W = c.w.W; p.ldw = c.w.ldw; p.Wh = c.w.Wh; p.ldh = c.w.ldh; p.R = c.R; p.ldr = c.ldr;
        p.m = c.m; p.c0 = c0; p.b = w; p.lowp = c.lowp == 2 ? 3 : c.lowp;
        p.rbuf = c.w.rbuf; p.qbuf = c.w.qbuf; p.cnt = c.w.cnt; p.err = c.w.err; p.leaf = c.leaf;
        LLS_TRY(panel_qr(p, c.st));
        if (c.lowp == 2) {
            // FP8: the copy of Q needs per-column scales (|q| ~ m^-1/2 is below E4M3's normal
            // range), so it is cast after the panel, column-major for the projection and
            // row-major for the update
            LLS_TRY(scale_cast_columns(c.w.W, c.w.ldw, c.m, c0, w, c.w.Wh, c.w.ldh, 2, c.w.sQ + c0, c.st));
            LLS_TRY(rowmajor_copy8(c.w.Wh, c.w.ldh, c.m, c0, w, c.w.QT, c.w.ldq, c.st));
        }
        return LLS_OK;
    }
    const int w1 = split_point(w, c.pw), w2 = w - w1;
    if (w1 == c.pw && w2 <= c.pw && (c.lowp == 0 || c.lowp == 1) && c.leaf == 0 && c.k.node_mode == 0) {
        // both halves are panels: left panel, node and right panel in one launch
        LLS_TRY(gate_upto(c, c0 + w));
        BlockCall bc;
        bc.W = c.w.W; bc.ldw = c.w.ldw; bc.Wh = c.w.Wh; bc.ldh = c.w.ldh; bc.R = c.R; bc.ldr = c.ldr;
        bc.m = c.m; bc.c0 = c0; bc.w1 = w1; bc.w2 = w2; bc.lowp = c.lowp;
        bc.rbuf = c.w.rbuf; bc.cnt = c.w.cnt; bc.part = c.w.part; bc.part_floats = c.w.part_floats;
        bc.err = c.w.err;
        const int r = block_fused_qr(bc, c.st);
        if (r != LLS_ERR_UNSUPPORTED) return r;
    }
    LLS_TRY(qr_rec(c, c0, w1));
    LLS_TRY(gate_upto(c, c0 + w));
    float* R12 = c.R + (size_t)c0 + (size_t)(c0 + w1) * c.ldr;
    float* A2 = c.w.W + (size_t)(c0 + w1) * c.w.ldw;
    const float* Q1 = c.w.W + (size_t)c0 * c.w.ldw;
    if (c.lowp == 3) {
        LLS_TRY(simt_projection_f32(Q1, A2, c.w.ldw, c.m, w1, w2, R12, c.ldr, c.w.part, c.st));
        LLS_TRY(simt_update_f32(Q1, c.w.ldw, R12, c.ldr, A2, c.m, w1, w2, c.st));
    } else {
        const size_t esz = c.lowp == 2 ? 1 : 2;
        const char* Whb = (const char*)c.w.Wh;
        if (c.k.node_mode <= 1) {
            NodeCall nc;
            nc.W = c.w.W; nc.ldw = c.w.ldw; nc.Wh = c.w.Wh; nc.ldh = c.w.ldh;
            nc.m = c.m; nc.c0 = c0; nc.w1 = w1; nc.w2 = w2; nc.lowp = c.lowp;
            nc.R = c.R; nc.ldr = c.ldr; nc.part = c.w.part; nc.part_floats = c.w.part_floats;
            nc.R12l = c.w.R12l; nc.f = c.w.f; nc.bar = c.w.nbar; nc.err = c.w.err;
            const int r = node_fused(nc, c.st);
            if (r != LLS_ERR_UNSUPPORTED) {
                LLS_TRY(r);
                return qr_rec(c, c0 + w1, w2);
            }
        }
        LLS_TRY(scale_cast_columns(c.w.W, c.w.ldw, c.m, c0 + w1, w2, c.w.Wh, c.w.ldh, c.lowp, c.w.eA, c.st));
        ProjCall pc;
        pc.Q1l = Whb + esz * (size_t)c0 * c.w.ldh;
        pc.A2l = Whb + esz * (size_t)(c0 + w1) * c.w.ldh;
        pc.ldh = c.w.ldh; pc.m = c.m; pc.w1 = w1; pc.w2 = w2; pc.e = c.w.eA;
        pc.R12 = R12; pc.ldr = c.ldr; pc.R12l = c.w.R12l; pc.f = c.w.f;
        pc.ldrl = (int)align_up((size_t)w1, c.lowp == 2 ? 16 : 8);      // 16-byte rows for TMA
        pc.sq = c.lowp == 2 ? c.w.sQ + c0 : nullptr;
        pc.part = c.w.part; pc.part_floats = c.w.part_floats; pc.lowp = c.lowp; pc.err = c.w.err;
        pc.gemm_kernel = c.k.gemm_kernel;
        LLS_TRY(gemm_projection(pc, c.st));
        UpdCall uc;
        uc.Q1l = pc.Q1l; uc.ldh = c.w.ldh; uc.R12l = c.w.R12l; uc.ldrl = pc.ldrl; uc.f = c.w.f; uc.err = c.w.err;
        uc.A2 = A2; uc.ldw = c.w.ldw; uc.m = c.m; uc.w1 = w1; uc.w2 = w2; uc.lowp = c.lowp;
        uc.gemm_kernel = c.k.gemm_kernel;
        if (c.lowp == 2) { uc.QT = c.w.QT + c0; uc.ldq = c.w.ldq; }
        LLS_TRY(gemm_update(uc, c.st));
    }
    return qr_rec(c, c0 + w1, w2);
}

// gate: null when A is copied into W here; otherwise W fills in chunks on another stream.
// anorm2: when non-null (and A is copied here), ||A||_F^2 is formed in the same pass as the copy.
static int run_qr(int m, int n, const float* A, int lda, float* R, int ldr, const lls_options& o,
                  const Knobs& k, QrWs& w, cudaStream_t st, ColumnGate* gate = nullptr, double* anorm2 = nullptr) {
    LLS_CUDA_TRY(cudaMemsetAsync(w.cnt, 0, sizeof(unsigned) * w.cnt_words, st));
    LLS_CUDA_TRY(cudaMemsetAsync(w.nbar, 0, sizeof(unsigned) * 4, st));
    LLS_CUDA_TRY(cudaMemsetAsync(w.err, 0, sizeof(int) * 16, st));
    if (!gate) {
        if (anorm2) LLS_TRY(copy_fro_sumsq(A, lda, w.W, w.ldw, m, n, w.red, anorm2, st));
        else LLS_TRY(copy_matrix(A, lda, w.W, w.ldw, m, n, st));
    }
    LLS_CUDA_TRY(cudaMemset2DAsync(R, sizeof(float) * (size_t)ldr, 0, sizeof(float) * (size_t)n, (size_t)n, st));
    QrCtx c;
    c.m = m; c.n = n; c.pw = o.panel_width; c.lowp = lowp_code(o.gemm_prec); c.leaf = o.panel_leaf;
    c.k = k;
    c.w = w; c.R = R; c.ldr = ldr; c.st = st; c.gate = gate;
    LLS_TRY(qr_rec(c, 0, n));
    LLS_TRY(gate_upto(c, n));
    if (o.reorth) {
        // A = Q1 R1 with Q1 in W; factor Q1 = Q2 R2 by the same recursion, so A = Q2 (R2 R1)
        LLS_CUDA_TRY(cudaMemcpy2DAsync(w.R1, sizeof(float) * (size_t)n, R, sizeof(float) * (size_t)ldr,
                                       sizeof(float) * (size_t)n, (size_t)n, cudaMemcpyDeviceToDevice, st));
        LLS_CUDA_TRY(cudaMemset2DAsync(R, sizeof(float) * (size_t)ldr, 0, sizeof(float) * (size_t)n, (size_t)n, st));
        LLS_TRY(qr_rec(c, 0, n));
        LLS_TRY(triu_product(R, ldr, w.R1, n, w.Rt, n, n, st));     // R2 R1
        LLS_CUDA_TRY(cudaMemcpy2DAsync(R, sizeof(float) * (size_t)ldr, w.Rt, sizeof(float) * (size_t)n,
                                       sizeof(float) * (size_t)n, (size_t)n, cudaMemcpyDeviceToDevice, st));
    }
    return LLS_OK;
}

}  // namespace lls

#include <atomic>

namespace lls {
extern std::atomic<unsigned long long> g_launches;
}  // namespace lls

using namespace lls;

// LLS_DEBUG builds: clear the translation units' index-check records before a public call
// and read them after it; the release build compiles both to nothing.
#define LLS_DEBUG_BEGIN(st) do { if (LLS_DEBUG) ::lls::debug_reset(st); } while (0)
static int debug_end(int status, cudaStream_t st) {
    if (!LLS_DEBUG) return status;
    const int d = ::lls::debug_collect(st);
    return d != LLS_OK ? d : status;
}

extern "C" {

unsigned long long lls_kernel_launch_count(void) { return g_launches.load(std::memory_order_relaxed); }

void lls_default_options(lls_options* o) {
    if (!o) return;
    memset(o, 0, sizeof(*o));
    o->gemm_prec = LLS_PREC_FP16;
    o->target = LLS_TARGET_FP64;
    o->tol = 0.0;
    o->max_iter = 200;
    o->panel_width = 0;        // auto: the recorded setting for the shape, else 16
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
        case LLS_ERR_TOO_LARGE: return "sizes exceed the fixed scratch of this entry point";
        case LLS_ERR_BOUNDS: return "index check failed (debug build)";
        default: return "unknown status";
    }
}

static size_t qr_ws_bytes(int m, int n, const lls_options& o) {
    WsArena ar(nullptr, SIZE_MAX);
    QrWs w;
    qr_layout(ar, m, n, o, w);
    return ar.off;
}

size_t qr_factor_workspace_size(int m, int n, const lls_options* opts) {
    lls_options o;
    resolve(opts, o);
    if (n < 1 || m < n || !valid_opts(o)) return 0;
    if (!auto_width(opts)) return qr_ws_bytes(m, n, o);
    size_t mx = 0;
    for (int pw : kTuneWidths) {
        lls_options c = o;
        c.panel_width = pw;
        if (!valid_opts(c)) continue;
        const size_t b = qr_ws_bytes(m, n, c);
        if (b > mx) mx = b;
    }
    return mx;
}

struct QrCall {
    int m, n, lda, ldq, ldr;
    const float* A; float* Q; float* R;
    lls_options o;
    Knobs k;
    QrWs w;
};

static int enqueue_qr(void* p, cudaStream_t st, cudaEvent_t*, bool) {
    QrCall& c = *(QrCall*)p;
    LLS_TRY(run_qr(c.m, c.n, c.A, c.lda, c.R, c.ldr, c.o, c.k, c.w, st));
    if (c.Q) LLS_TRY(copy_matrix(c.w.W, c.w.ldw, c.Q, c.ldq, c.m, c.n, st));
    return poison_diag_on_error(c.R, c.ldr, c.n, c.w.err, st);   // a wait that gave up: NaN diagonal
}

static int current_device() {
    int d = 0;
    cudaGetDevice(&d);
    return d;
}

static int qr_factor_impl(int m, int n, const float* A, int lda, float* Q, int ldq, float* R, int ldr,
              void* ws, size_t ws_bytes, const lls_options* opts, cudaStream_t stream) {
    lls_options o;
    Knobs k;
    resolve_settings(opts, 0, m, n, o, k);
    if (n < 1 || m < n || lda < m || ldr < n || !A || !R || !ws) return LLS_ERR_ARG;
    if (Q && ldq < m) return LLS_ERR_ARG;
    if (!valid_opts(o)) return LLS_ERR_ARG;
    if (((uintptr_t)ws & 255) != 0) return LLS_ERR_WORKSPACE;
    WsArena ar(ws, ws_bytes);
    QrCall c;
    qr_layout(ar, m, n, o, c.w);
    if (!ar.ok) return LLS_ERR_WORKSPACE;
    c.m = m; c.n = n; c.lda = lda; c.ldq = ldq; c.ldr = ldr; c.A = A; c.Q = Q; c.R = R; c.o = o; c.k = k;
    GraphKey key;
    memset(&key, 0, sizeof(key));
    key.op = 1; key.device = current_device();
    key.ints[0] = m; key.ints[1] = n; key.ints[2] = lda; key.ints[3] = Q ? ldq : 0; key.ints[4] = ldr;
    key.ptrs[0] = A; key.ptrs[1] = Q; key.ptrs[2] = R; key.ptrs[3] = ws;
    key.ws_bytes = ws_bytes; key.opts = o; key.knobs = k;
    trace_mark(stream);
    LLS_TRY(run_graphed(key, stream, enqueue_qr, &c, nullptr));
    trace_flush();
    return LLS_OK;
}

size_t lls_lowp_projection_workspace_size(int m, int w1, int w2) {
    if (m < 1 || w1 < 1 || w2 < 1) return 0;
    return align_up(sizeof(float) * proj_partial_floats(m, w1, w2), 256) + 256;
}

static int lls_lowp_projection_impl(int m, int w1, int w2, int prec, const void* Q1l, const void* A2l, int ldh,
                        const int* e, float* R12, int ldr, void* R12l, int ldrl, int* f, void* ws,
                        size_t ws_bytes, cudaStream_t stream) {
    if (m < 1 || w1 < 1 || w2 < 1 || ldh < m || ldr < w1 || ldrl < w1 || (ldrl & 7) != 0) return LLS_ERR_ARG;
    if (prec != LLS_PREC_FP16 && prec != LLS_PREC_BF16) return LLS_ERR_ARG;
    if (!Q1l || !A2l || !e || !R12 || !R12l || !f || !ws) return LLS_ERR_ARG;
    if (((uintptr_t)ws & 255) != 0) return LLS_ERR_WORKSPACE;
    WsArena ar(ws, ws_bytes);
    ProjCall pc;
    pc.part_floats = proj_partial_floats(m, w1, w2);
    pc.part = ar.take<float>(pc.part_floats);
    pc.err = ar.take<int>(16);
    if (!ar.ok) return LLS_ERR_WORKSPACE;
    LLS_CUDA_TRY(cudaMemsetAsync(pc.err, 0, sizeof(int) * 16, stream));
    pc.Q1l = Q1l; pc.A2l = A2l; pc.ldh = ldh; pc.m = m; pc.w1 = w1; pc.w2 = w2; pc.e = e;
    pc.R12 = R12; pc.ldr = ldr; pc.R12l = R12l; pc.ldrl = ldrl; pc.f = f; pc.lowp = lowp_code(prec);
    return gemm_projection(pc, stream);
}

static int lls_lowp_update_impl(int m, int w1, int w2, int prec, const void* Q1l, int ldh, const void* R12l,
                    int ldrl, const int* f, float* A2, int lda, void* ws, size_t ws_bytes,
                    cudaStream_t stream) {
    if (m < 1 || w1 < 1 || w2 < 1 || ldh < m || lda < m || ldrl < w1 || (ldrl & 7) != 0) return LLS_ERR_ARG;
    if (prec != LLS_PREC_FP16 && prec != LLS_PREC_BF16) return LLS_ERR_ARG;
    if (!Q1l || !R12l || !f || !A2 || !ws) return LLS_ERR_ARG;
    if (((uintptr_t)ws & 255) != 0 || ws_bytes < 256) return LLS_ERR_WORKSPACE;
    UpdCall uc;
    uc.err = (int*)ws;
    LLS_CUDA_TRY(cudaMemsetAsync(uc.err, 0, sizeof(int) * 16, stream));
    uc.Q1l = Q1l; uc.ldh = ldh; uc.R12l = R12l; uc.ldrl = ldrl; uc.f = f; uc.A2 = A2; uc.ldw = lda;
    uc.m = m; uc.w1 = w1; uc.w2 = w2; uc.lowp = lowp_code(prec);
    return gemm_update(uc, stream);
}

struct PanelWs {
    float* rbuf; float* qbuf; unsigned* cnt; size_t cnt_words; int* err;
};

static void panel_layout(WsArena& ar, int m, PanelWs& w) {
    size_t rb, qb, cw;
    panel_scratch_sizes(m, rb, qb, cw);
    w.rbuf = ar.take<float>(rb);
    w.qbuf = ar.take<float>(qb);
    w.cnt = ar.take<unsigned>(cw);
    w.cnt_words = cw;
    w.err = ar.take<int>(16);
}

size_t lls_panel_qr_workspace_size(int m, int b) {
    if (m < 1 || b < 1 || b > 32 || m < b) return 0;
    WsArena ar(nullptr, ~(size_t)0);
    PanelWs w;
    panel_layout(ar, m, w);
    return ar.off;
}

static int lls_panel_qr_impl(int m, int b, int prec, float* W, int ldw, void* Wh, int ldh, float* R, int ldr, void* ws,
                 size_t ws_bytes, cudaStream_t stream) {
    if (m < 1 || b < 1 || b > 32 || m < b || ldw < m || ldr < b || !W || !R || !ws) return LLS_ERR_ARG;
    if (prec != LLS_PREC_FP16 && prec != LLS_PREC_BF16 && prec != LLS_PREC_FP32) return LLS_ERR_ARG;
    if (prec != LLS_PREC_FP32 && (!Wh || ldh < m)) return LLS_ERR_ARG;
    if (((uintptr_t)ws & 255) != 0) return LLS_ERR_WORKSPACE;
    WsArena ar(ws, ws_bytes);
    PanelWs w;
    panel_layout(ar, m, w);
    if (!ar.ok) return LLS_ERR_WORKSPACE;
    // counters and error word are zero on entry (caller's zero fill, then self-resetting)
    PanelCall p;
    p.W = W; p.ldw = ldw; p.Wh = prec == LLS_PREC_FP32 ? nullptr : Wh; p.ldh = ldh; p.R = R; p.ldr = ldr;
    p.m = m; p.c0 = 0; p.b = b; p.lowp = lowp_code(prec);
    p.rbuf = w.rbuf; p.qbuf = w.qbuf; p.cnt = w.cnt; p.err = w.err;
    return panel_qr(p, stream);
}

struct BlockWs {
    PanelWs p; float* part;
};

static void block_layout(WsArena& ar, int m, BlockWs& w) {
    panel_layout(ar, m, w.p);
    w.part = ar.take<float>(block_fused_part_floats());
}

size_t lls_panel_block_qr_workspace_size(int m, int w1, int w2) {
    if (m < 1 || w1 < 1 || w2 < 1 || m < w1 + w2) return 0;
    WsArena ar(nullptr, ~(size_t)0);
    BlockWs w;
    block_layout(ar, m, w);
    return ar.off;
}

static int lls_panel_block_qr_impl(int m, int w1, int w2, int prec, float* W, int ldw, void* Wh, int ldh, float* R,
                       int ldr, void* ws, size_t ws_bytes, cudaStream_t stream) {
    if (w1 < 1 || w2 < 1 || m < w1 + w2 || ldw < m || ldh < m || ldr < w1 + w2) return LLS_ERR_ARG;
    if (!W || !Wh || !R || !ws) return LLS_ERR_ARG;
    if (prec != LLS_PREC_FP16 && prec != LLS_PREC_BF16) return LLS_ERR_ARG;
    if (((uintptr_t)ws & 255) != 0) return LLS_ERR_WORKSPACE;
    WsArena ar(ws, ws_bytes);
    BlockWs w;
    block_layout(ar, m, w);
    if (!ar.ok) return LLS_ERR_WORKSPACE;
    BlockCall bc;
    bc.W = W; bc.ldw = ldw; bc.Wh = Wh; bc.ldh = ldh; bc.R = R; bc.ldr = ldr;
    bc.m = m; bc.c0 = 0; bc.w1 = w1; bc.w2 = w2; bc.lowp = lowp_code(prec);
    bc.rbuf = w.p.rbuf; bc.cnt = w.p.cnt; bc.part = w.part; bc.part_floats = block_fused_part_floats();
    bc.err = w.p.err;
    if (!block_fused_supported(bc)) return LLS_ERR_UNSUPPORTED;
    const size_t wt = (size_t)(w1 + w2);
    LLS_CUDA_TRY(cudaMemset2DAsync(R, sizeof(float) * (size_t)ldr, 0, sizeof(float) * wt, wt, stream));
    return block_fused_qr(bc, stream);
}

static void lls_layout(WsArena& ar, int m, int n, const lls_options& o, QrWs& w, float*& R,
                       float*& Minv, float*& Mt, float*& tmp, void*& ks, size_t& ks_bytes, double*& hist) {
    qr_layout(ar, m, n, o, w);
    R = ar.take<float>((size_t)n * n);
    Minv = ar.take<float>((size_t)n * n);
    Mt = ar.take<float>((size_t)n * n);
    tmp = ar.take<float>((size_t)n * n);
    ks_bytes = krylov_scratch_bytes(m, n, 0, o.krylov == LLS_KRYLOV_CGLS);
    const size_t ds = direct_start_scratch_bytes(m, n);   // the direct start borrows the Krylov scratch
    if (ks_bytes < ds) ks_bytes = ds;
    ks = ar.take<char>(ks_bytes);
    hist = ar.take<double>(kHistLen + kPhaseLen);   // the history, then the CGLS phase log
}

static size_t solve_ws_bytes(int m, int n, const lls_options& o) {
    WsArena ar(nullptr, SIZE_MAX);
    QrWs w; float *R, *Mi, *Mt, *tmp; void* ks; size_t kb; double* hist;
    lls_layout(ar, m, n, o, w, R, Mi, Mt, tmp, ks, kb, hist);
    return ar.off;
}

// The workspace of a solve: for "auto" options, enough for every panel width a tuning may pick.
static size_t solve_ws_bytes_auto(int m, int n, const lls_options* opts, const lls_options& o) {
    if (!auto_width(opts)) return solve_ws_bytes(m, n, o);
    size_t mx = 0;
    for (int pw : kTuneWidths) {
        lls_options c = o;
        c.panel_width = pw;
        if (!valid_opts(c)) continue;
        const size_t b = solve_ws_bytes(m, n, c);
        if (b > mx) mx = b;
    }
    return mx;
}

size_t lls_solve_workspace_size(int m, int n, const lls_options* opts) {
    lls_options o;
    resolve(opts, o);
    if (n < 1 || m < n || !valid_opts(o)) return 0;
    return solve_ws_bytes_auto(m, n, opts, o);
}

struct SolveCall {
    int m, n, lda, ldr;
    const float* A; const double* b; double* x; float* R_out;
    lls_options o;
    Knobs k;
    QrWs w;
    float *R, *Minv, *Mt, *tmp;
    void* ks; size_t kb;
    double* hist;
};

// The solve on `st`; gate non-null when W fills in chunks on another stream (host input).
// LLS_LOG=1: the Krylov stop quantity of every iteration on stderr; LLS_LOG=2 adds the median
// time of each phase of the CGLS iteration (between consecutive grid barriers, seen by CTA 0).
static int log_level() {
    static const int lv = [] {
        const char* v = getenv("LLS_LOG");
        if (!v || !v[0] || v[0] == '0') return 0;
        return v[0] == '2' ? 2 : 1;
    }();
    return lv;
}

static int solve_body(SolveCall& c, cudaStream_t st, cudaEvent_t* ev, bool capturing, ColumnGate* gate) {
    const int m = c.m, n = c.n;
    if (ev) record_phase(ev[0], st, capturing);
    LLS_CUDA_TRY(cudaMemsetAsync(c.w.dinfo, 0, sizeof(double) * 16, st));
    // without a gate A is copied into W here, and its norm comes with the copy
    LLS_TRY(run_qr(m, n, c.A, c.lda, c.R, n, c.o, c.k, c.w, st, gate, gate ? nullptr : c.w.dinfo + 8));
    if (c.R_out) LLS_TRY(copy_matrix(c.R, n, c.R_out, c.ldr, n, n, st));
    LLS_TRY(check_diag(c.R, n, n, c.w.err, st));
    LLS_TRY(tri_inverse(c.R, n, n, c.o.panel_width, c.Minv, c.Mt, c.tmp, c.w.err, st));
    // the host-operand solve copies A in chunks: its norm is formed here, with the same sums
    if (gate) LLS_TRY(copy_fro_sumsq(c.A, c.lda, nullptr, 0, m, n, c.w.red, c.w.dinfo + 8, st));
    LLS_TRY(fro_sumsq(c.Minv, n, n, n, c.w.red + 4096, c.w.dinfo + 9, st));
    if (c.o.x0 == LLS_X0_DIRECT)   // x0 = R^{-1} Q^T b from the factors; W holds Q
        LLS_TRY(direct_start(c.w.W, c.w.ldw, m, n, c.b, c.Mt, c.x, c.ks, c.kb, st));
    if (ev) record_phase(ev[1], st, capturing);
    KrylovCall kc;
    kc.m = m; kc.n = n; kc.A = c.A; kc.lda = c.lda; kc.b = c.b; kc.x = c.x; kc.Minv = c.Minv; kc.Mt = c.Mt;
    kc.method = c.o.krylov; kc.target = c.o.target; kc.tol = c.o.tol; kc.max_iter = c.o.max_iter;
    kc.scratch = c.ks; kc.scratch_bytes = c.kb; kc.dev_err = c.w.err; kc.dev_info = c.w.dinfo;
    kc.x_zero = c.o.x0 == LLS_X0_ZERO ? 1 : 0;
    kc.hist = c.hist;
    if (c.hist && log_level() >= 2) {
        kc.phases = reinterpret_cast<unsigned long long*>(c.hist + kHistLen);
        LLS_CUDA_TRY(cudaMemsetAsync(kc.phases, 0, sizeof(unsigned long long) * kPhaseLen, st));
    }
    kc.ctas = c.k.krylov_ctas;
    LLS_TRY(krylov_solve(kc, st));
    if (ev) record_phase(ev[2], st, capturing);
    return LLS_OK;
}

static int enqueue_solve(void* p, cudaStream_t st, cudaEvent_t* ev, bool capturing) {
    return solve_body(*(SolveCall*)p, st, ev, capturing, nullptr);
}


// LLS_LOG=2: per phase of the CGLS iteration, the median over the logged iterations of the time
// from one grid barrier to the next (phase 1 starts at the top of the iteration), in us. The
// log holds a stamp per grid barrier of CTA 0, iteration tops marked by the top bit.
static void print_phases(const unsigned long long* ph_dev, cudaStream_t stream) {
    std::vector<unsigned long long> t((size_t)kPhaseLen);
    if (cudaMemcpyAsync(t.data(), ph_dev, sizeof(unsigned long long) * kPhaseLen, cudaMemcpyDeviceToHost,
                        stream) != cudaSuccess ||
        cudaStreamSynchronize(stream) != cudaSuccess)
        return;
    constexpr unsigned long long kTop = 1ull << 63;
    constexpr int P = 8;   // grid barriers per iteration of the two-pass engine
    std::vector<std::vector<double>> d(P);
    std::vector<double> tot;
    for (int i = 0; i + P < kPhaseLen; ++i) {
        if (!(t[(size_t)i] & kTop)) continue;
        bool ok = true;
        for (int k = 1; k <= P && ok; ++k) {
            const unsigned long long a = t[(size_t)i + k - 1] & ~kTop, b = t[(size_t)i + k];
            ok = !(b & kTop) && b > a;
        }
        if (!ok) continue;   // an iteration that ended early (stop test) or was not reached
        for (int k = 1; k <= P; ++k)
            d[(size_t)k - 1].push_back((double)(t[(size_t)i + k] - (t[(size_t)i + k - 1] & ~kTop)) * 1e-3);
        tot.push_back((double)(t[(size_t)i + P] - (t[(size_t)i] & ~kTop)) * 1e-3);
    }
    if (tot.empty()) return;
    auto med = [](std::vector<double> v) {
        std::sort(v.begin(), v.end());
        return v[v.size() / 2];
    };
    fprintf(stderr, "[lls log] CGLS phases, median us over %zu iterations:", tot.size());
    for (int k = 0; k < P; ++k) fprintf(stderr, " %d:%.1f", k + 1, med(d[(size_t)k]));
    fprintf(stderr, " total:%.1f\n", med(tot));
}

// LLS_LOG=1: the stop quantity of every iteration (eta_est for the FP64 target, the forward
// error estimate for the FP32 target) to stderr, one line per solve.
static void print_history(const double* hist_dev, int iters, int m, int n, cudaStream_t stream) {
    const int count = (iters + 1 < kHistLen ? iters + 1 : kHistLen);
    std::vector<double> h((size_t)count);
    if (cudaMemcpyAsync(h.data(), hist_dev, sizeof(double) * (size_t)count, cudaMemcpyDeviceToHost, stream) !=
            cudaSuccess ||
        cudaStreamSynchronize(stream) != cudaSuccess)
        return;
    fprintf(stderr, "[lls log] m=%d n=%d iterations=%d stop quantity per iteration:", m, n, iters);
    for (int k = 0; k < count; ++k) fprintf(stderr, " %d:%.3e", k, h[(size_t)k]);
    fprintf(stderr, "\n");
}

// Reads the device info record and error word after the solve (synchronizes the stream) and
// fills info; returns the solve's status.
static int finish_info(const QrWs& w, cudaEvent_t* ev, lls_info* info, cudaStream_t stream,
                       const double* hist = nullptr, int m = 0, int n = 0) {
    double hinfo[16];
    int herr = 0;
    LLS_CUDA_TRY(cudaMemcpyAsync(hinfo, w.dinfo, sizeof(hinfo), cudaMemcpyDeviceToHost, stream));
    LLS_CUDA_TRY(cudaMemcpyAsync(&herr, w.err, sizeof(int), cudaMemcpyDeviceToHost, stream));
    LLS_CUDA_TRY(cudaStreamSynchronize(stream));
    if (hist && log_level() >= 1) print_history(hist, (int)hinfo[0], m, n, stream);
    if (hist && log_level() >= 2) print_phases(reinterpret_cast<const unsigned long long*>(hist + kHistLen), stream);
    cudaEventElapsedTime(&info->qr_ms, ev[0], ev[1]);
    cudaEventElapsedTime(&info->krylov_ms, ev[1], ev[2]);
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

// lls_solve with resolved options and implementation choices (also the autotuner's trial).
static int solve_core(int m, int n, const float* A, int lda, const double* b, double* x, float* R_out, int ldr,
                      void* ws, size_t ws_bytes, const lls_options& o, const Knobs& k, lls_info* info,
                      cudaStream_t stream) {
    if (info) memset(info, 0, sizeof(*info));
    if (n < 1 || m < n || lda < m || !A || !b || !x || !ws) return LLS_ERR_ARG;
    if (R_out && ldr < n) return LLS_ERR_ARG;
    if (!valid_opts(o)) return LLS_ERR_ARG;
    // CGLS and LSQR share the workspace layout and the stop tests
    if (((uintptr_t)ws & 255) != 0) return LLS_ERR_WORKSPACE;
    WsArena ar(ws, ws_bytes);
    SolveCall c;
    lls_layout(ar, m, n, o, c.w, c.R, c.Minv, c.Mt, c.tmp, c.ks, c.kb, c.hist);
    if (!ar.ok) return LLS_ERR_WORKSPACE;
    c.m = m; c.n = n; c.lda = lda; c.ldr = ldr; c.A = A; c.b = b; c.x = x; c.R_out = R_out; c.o = o; c.k = k;
    GraphKey key;
    memset(&key, 0, sizeof(key));
    key.op = 2; key.device = current_device();
    key.ints[0] = m; key.ints[1] = n; key.ints[2] = lda; key.ints[3] = R_out ? ldr : 0;
    key.ptrs[0] = A; key.ptrs[1] = b; key.ptrs[2] = x; key.ptrs[3] = R_out; key.ptrs[4] = ws;
    key.ws_bytes = ws_bytes; key.opts = o; key.knobs = k;

    cudaEvent_t own[3] = {nullptr, nullptr, nullptr};
    cudaEvent_t ev[3] = {nullptr, nullptr, nullptr};
    if (info) {
        for (int i = 0; i < 3; ++i) LLS_CUDA_TRY(cudaEventCreate(&own[i]));
        for (int i = 0; i < 3; ++i) ev[i] = own[i];
    }
    trace_mark(stream);
    int rc = run_graphed(key, stream, enqueue_solve, &c, info ? ev : nullptr);
    trace_flush();
    if (rc != LLS_OK || !info) {
        for (auto& e : own) if (e) cudaEventDestroy(e);
        return rc;
    }
    rc = finish_info(c.w, ev, info, stream, c.hist, m, n);
    for (auto& e : own) cudaEventDestroy(e);
    return rc;
}

static int lls_solve_impl(int m, int n, const float* A, int lda, const double* b, double* x, float* R_out,
              int ldr, void* ws, size_t ws_bytes, const lls_options* opts, lls_info* info,
              cudaStream_t stream) {
    lls_options o;
    Knobs k;
    resolve_settings(opts, 0, m, n, o, k);
    return solve_core(m, n, A, lda, b, x, R_out, ldr, ws, ws_bytes, o, k, info, stream);
}


// ---------------------------------------------------------------------------------------
// The solve from page-locked host buffers. A goes up in column chunks of doubling width
// (64, 64, 128, 256, ... columns) on a side stream, each chunk into a device copy of A and
// into W; the recursion waits for a chunk just before it first touches the chunk's columns,
// so all but the first chunk's upload overlaps the factorization. x comes back at the end.

struct HostRes {
    cudaStream_t side = nullptr;
    cudaEvent_t fork = nullptr;
    cudaEvent_t ev[kMaxChunks];
};
static std::mutex g_host_mu;            // one enqueue at a time: the events are shared
static HostRes g_host_res[64];

static int host_res(HostRes*& r) {
    int dev = 0;
    LLS_CUDA_TRY(cudaGetDevice(&dev));
    if (dev < 0 || dev >= 64) return LLS_ERR_UNSUPPORTED;
    HostRes& h = g_host_res[dev];
    if (!h.side) {
        LLS_CUDA_TRY(cudaStreamCreateWithFlags(&h.side, cudaStreamNonBlocking));
        LLS_CUDA_TRY(cudaEventCreateWithFlags(&h.fork, cudaEventDisableTiming));
        for (auto& e : h.ev) LLS_CUDA_TRY(cudaEventCreateWithFlags(&e, cudaEventDisableTiming));
    }
    r = &h;
    return LLS_OK;
}

static void plan_chunks(int n, ColumnGate& g) {
    g.count = 0;
    g.ready = 0;
    int c = 0;
    while (c < n && g.count < kMaxChunks) {
        g.start[g.count++] = c;
        c = c == 0 ? 64 : (c > n / 2 ? n : 2 * c);
        if (c > n) c = n;
    }
    g.start[g.count] = n;
}

struct HostSolveCall {
    SolveCall s;                        // the device solve on the workspace's copies of A, b, x
    const float* Ah; int ldah;
    const double* bh; double* xh;
};

static void host_layout(WsArena& ar, int m, int n, int& lda, float*& A, double*& b, double*& x) {
    lda = (int)align_up((size_t)m, 64);
    A = ar.take<float>((size_t)lda * n);
    b = ar.take<double>((size_t)m);
    x = ar.take<double>((size_t)n);
}

static int enqueue_solve_host(void* p, cudaStream_t st, cudaEvent_t* ev, bool capturing) {
    HostSolveCall& h = *(HostSolveCall*)p;
    SolveCall& c = h.s;
    const int m = c.m, n = c.n;
    HostRes* r = nullptr;
    LLS_TRY(host_res(r));
    ColumnGate g;
    plan_chunks(n, g);
    for (int k = 0; k < g.count; ++k) g.ev[k] = r->ev[k];
    LLS_CUDA_TRY(cudaEventRecord(r->fork, st));
    LLS_CUDA_TRY(cudaStreamWaitEvent(r->side, r->fork, 0));
    float* Ad = const_cast<float*>(c.A);
    LLS_CUDA_TRY(cudaMemcpyAsync(const_cast<double*>(c.b), h.bh, sizeof(double) * (size_t)m,
                                 cudaMemcpyHostToDevice, r->side));
    if (c.o.x0 == LLS_X0_GIVEN)   // the starting x comes from the caller's host x
        LLS_CUDA_TRY(cudaMemcpyAsync(c.x, h.xh, sizeof(double) * (size_t)n, cudaMemcpyHostToDevice, r->side));
    for (int k = 0; k < g.count; ++k) {
        const int c0 = g.start[k], cols = g.start[k + 1] - c0;
        LLS_CUDA_TRY(cudaMemcpy2DAsync(Ad + (size_t)c0 * c.lda, sizeof(float) * (size_t)c.lda,
                                       h.Ah + (size_t)c0 * h.ldah, sizeof(float) * (size_t)h.ldah,
                                       sizeof(float) * (size_t)m, (size_t)cols, cudaMemcpyHostToDevice, r->side));
        LLS_CUDA_TRY(cudaMemcpy2DAsync(c.w.W + (size_t)c0 * c.w.ldw, sizeof(float) * (size_t)c.w.ldw,
                                       Ad + (size_t)c0 * c.lda, sizeof(float) * (size_t)c.lda,
                                       sizeof(float) * (size_t)m, (size_t)cols, cudaMemcpyDeviceToDevice, r->side));
        LLS_CUDA_TRY(cudaEventRecord(g.ev[k], r->side));
    }
    LLS_TRY(solve_body(c, st, ev, capturing, &g));   // joins every chunk before A's norm and the Krylov phase
    LLS_CUDA_TRY(cudaMemcpyAsync(h.xh, c.x, sizeof(double) * (size_t)n, cudaMemcpyDeviceToHost, st));
    return LLS_OK;
}

int lls_upload_chunks(int n, int* start, int max_entries) {
    if (n < 1 || !start || max_entries < 2) return LLS_ERR_ARG;
    ColumnGate g;
    plan_chunks(n, g);
    if (g.count + 1 > max_entries) return LLS_ERR_ARG;
    for (int k = 0; k <= g.count; ++k) start[k] = g.start[k];
    return g.count;
}

static bool page_locked(const void* p) {
    cudaPointerAttributes a;
    if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return a.type == cudaMemoryTypeHost;
}

size_t lls_solve_host_workspace_size(int m, int n, const lls_options* opts) {
    lls_options o;
    resolve(opts, o);
    if (n < 1 || m < n || !valid_opts(o)) return 0;
    WsArena ar(nullptr, SIZE_MAX);
    ar.off = align_up(solve_ws_bytes_auto(m, n, opts, o), 256);
    int lda; float* A; double *b, *x;
    host_layout(ar, m, n, lda, A, b, x);
    return ar.off;
}

static int lls_solve_host_impl(int m, int n, const float* A, int lda, const double* b, double* x, void* ws,
                   size_t ws_bytes, const lls_options* opts, lls_info* info, cudaStream_t stream) {
    lls_options o;
    Knobs k;
    resolve_settings(opts, 0, m, n, o, k);
    if (info) memset(info, 0, sizeof(*info));
    if (n < 1 || m < n || lda < m || !A || !b || !x || !ws) return LLS_ERR_ARG;
    if (!valid_opts(o)) return LLS_ERR_ARG;
    if (!page_locked(A) || !page_locked(b) || !page_locked(x)) return LLS_ERR_ARG;
    if (((uintptr_t)ws & 255) != 0) return LLS_ERR_WORKSPACE;
    // the device solve's share of the workspace is the one an "auto" call sizes
    const size_t solve_share = align_up(solve_ws_bytes_auto(m, n, opts, o), 256);
    if (ws_bytes < solve_share) return LLS_ERR_WORKSPACE;
    WsArena ar(ws, solve_share);
    HostSolveCall h;
    SolveCall& c = h.s;
    lls_layout(ar, m, n, o, c.w, c.R, c.Minv, c.Mt, c.tmp, c.ks, c.kb, c.hist);
    if (!ar.ok) return LLS_ERR_WORKSPACE;
    WsArena ar2((char*)ws + solve_share, ws_bytes - solve_share);
    int ldad; float* Ad; double *bd, *xd;
    host_layout(ar2, m, n, ldad, Ad, bd, xd);
    if (!ar2.ok) return LLS_ERR_WORKSPACE;
    c.m = m; c.n = n; c.lda = ldad; c.ldr = 0; c.A = Ad; c.b = bd; c.x = xd; c.R_out = nullptr; c.o = o; c.k = k;
    h.Ah = A; h.ldah = lda; h.bh = b; h.xh = x;
    GraphKey key;
    memset(&key, 0, sizeof(key));
    key.op = 4; key.device = current_device();
    key.ints[0] = m; key.ints[1] = n; key.ints[2] = lda;
    key.ptrs[0] = A; key.ptrs[1] = b; key.ptrs[2] = x; key.ptrs[3] = ws;
    key.ws_bytes = ws_bytes; key.opts = o; key.knobs = k;

    cudaEvent_t own[3] = {nullptr, nullptr, nullptr};
    cudaEvent_t ev[3] = {nullptr, nullptr, nullptr};
    if (info) {
        for (int i = 0; i < 3; ++i) LLS_CUDA_TRY(cudaEventCreate(&own[i]));
        for (int i = 0; i < 3; ++i) ev[i] = own[i];
    }
    int rc;
    {
        std::lock_guard<std::mutex> lk(g_host_mu);
        trace_mark(stream);
        rc = run_graphed(key, stream, enqueue_solve_host, &h, info ? ev : nullptr);
        trace_flush();
    }
    if (rc == LLS_OK && info) rc = finish_info(c.w, ev, info, stream, c.hist, m, n);
    for (auto& e : own) if (e) cudaEventDestroy(e);
    return rc;
}

// ---------------------------------------------------------------------------------------
// Adjoint of the least-squares solve (batched over independent problems).
// ---------------------------------------------------------------------------------------
struct BwdWs {
    float *Minv, *Mt, *tmp;
    double* z;
    void* ks; size_t kb;
    int* err; double* dinfo;
};

static void bwd_layout(WsArena& ar, int mmax, int nmax, BwdWs& w) {
    w.Minv = ar.take<float>((size_t)nmax * nmax);
    w.Mt = ar.take<float>((size_t)nmax * nmax);
    w.tmp = ar.take<float>((size_t)nmax * nmax);
    w.z = ar.take<double>(nmax);
    w.kb = krylov_scratch_bytes(mmax, nmax, 0);
    w.ks = ar.take<char>(w.kb);
    w.err = ar.take<int>(16);
    w.dinfo = ar.take<double>(16);
}

static bool batch_dims(int batch, const int* m, const int* n, int& mmax, int& nmax) {
    if (batch < 1 || !m || !n) return false;
    mmax = 0; nmax = 0;
    for (int i = 0; i < batch; ++i) {
        if (n[i] < 1 || m[i] < n[i]) return false;
        if (m[i] > mmax) mmax = m[i];
        if (n[i] > nmax) nmax = n[i];
    }
    return true;
}

// Batches of two or more problems that the batched kernels take run as one persistent launch;
// single problems and larger ones run problem after problem on the whole GPU.
static bool backward_batched(int batch, const int* m, const int* n) {
    if (batch < 2) return false;
    for (int i = 0; i < batch; ++i)
        if (!batched_supported(m[i], n[i])) return false;
    return true;
}

size_t lls_backward_workspace_size(int batch, const int* m, const int* n, const lls_options* opts) {
    lls_options o;
    resolve(opts, o);
    int mmax, nmax;
    if (!batch_dims(batch, m, n, mmax, nmax) || !valid_opts(o)) return 0;
    if (backward_batched(batch, m, n)) return batched_adjoint_workspace_bytes(batch, m, n);
    WsArena ar(nullptr, SIZE_MAX);
    BwdWs w;
    bwd_layout(ar, mmax, nmax, w);
    return ar.off;
}

static int lls_backward_impl(int batch, const int* m, const int* n, const float* const* A, const int* lda,
                 const double* const* b, const double* const* x, const float* const* R, const int* ldr,
                 const double* const* grad_x, float* const* grad_A, const int* ldga,
                 double* const* grad_b, void* ws, size_t ws_bytes, const lls_options* opts,
                 cudaStream_t stream) {
    lls_options o;
    resolve(opts, o);
    int mmax, nmax;
    if (!batch_dims(batch, m, n, mmax, nmax) || !valid_opts(o)) return LLS_ERR_ARG;
    if (!A || !lda || !b || !x || !R || !ldr || !grad_x || !grad_A || !ldga || !grad_b || !ws) return LLS_ERR_ARG;
    for (int i = 0; i < batch; ++i) {
        if (!A[i] || !b[i] || !x[i] || !R[i] || !grad_x[i] || !grad_A[i] || !grad_b[i]) return LLS_ERR_ARG;
        if (lda[i] < m[i] || ldr[i] < n[i] || ldga[i] < m[i]) return LLS_ERR_ARG;
    }
    if (((uintptr_t)ws & 255) != 0) return LLS_ERR_WORKSPACE;
    const double tol = o.target == LLS_TARGET_FP32 ? 1e-7 : 1e-13;
    trace_mark(stream);
    if (backward_batched(batch, m, n)) {
        const int r = batched_adjoint(batch, m, n, A, lda, b, x, R, ldr, grad_x, grad_A, ldga, grad_b, ws,
                                      ws_bytes, tol, o.max_iter, stream);
        trace_flush();
        return r;
    }
    WsArena ar(ws, ws_bytes);
    BwdWs w;
    bwd_layout(ar, mmax, nmax, w);
    if (!ar.ok) return LLS_ERR_WORKSPACE;
    LLS_CUDA_TRY(cudaMemsetAsync(w.err, 0, sizeof(int) * 16, stream));
    for (int i = 0; i < batch; ++i) {
        LLS_TRY(tri_inverse(R[i], ldr[i], n[i], o.panel_width, w.Minv, w.Mt, w.tmp, w.err, stream));
        AdjointCall c;
        c.m = m[i]; c.n = n[i]; c.A = A[i]; c.lda = lda[i]; c.b = b[i]; c.x = x[i]; c.g = grad_x[i];
        c.Minv = w.Minv; c.Mt = w.Mt; c.z = w.z; c.gA = grad_A[i]; c.ldga = ldga[i]; c.gb = grad_b[i];
        c.tol = tol;
        c.max_iter = o.max_iter;
        c.scratch = w.ks; c.scratch_bytes = w.kb; c.dev_err = w.err; c.dev_info = w.dinfo;
        LLS_TRY(adjoint_solve(c, stream));
    }
    trace_flush();
    return LLS_OK;
}

// ---------------------------------------------------------------------------------------
// Batched solve: many independent problems, one persistent launch (batched.cu).
// ---------------------------------------------------------------------------------------
struct BatchExec {
    int batch; const int* m; const int* n; void* ws; lls_options o; Knobs k;
};

static int enqueue_batched(void* p, cudaStream_t st, cudaEvent_t* ev, bool capturing) {
    BatchExec& c = *(BatchExec*)p;
    if (ev) record_phase(ev[0], st, capturing);
    LLS_TRY(batched_execute(c.batch, c.m, c.n, c.ws, c.o, c.k.batched_ctas, st));
    if (ev) { record_phase(ev[1], st, capturing); record_phase(ev[2], st, capturing); }
    return LLS_OK;
}

size_t lls_solve_batched_workspace_size(int batch, const int* m, const int* n, const lls_options* opts) {
    lls_options o;
    resolve(opts, o);
    int mmax, nmax;
    if (!batch_dims(batch, m, n, mmax, nmax) || !valid_opts(o)) return 0;
    for (int i = 0; i < batch; ++i)
        if (!batched_supported(m[i], n[i])) return 0;
    return batched_workspace_bytes(batch, m, n);
}

static int batched_core(int batch, const int* m, const int* n, const float* const* A, const int* lda,
                        const double* const* b, double* const* x, float* const* R_out, const int* ldr,
                        void* ws, size_t ws_bytes, const lls_options& o, const Knobs& k, lls_info* infos,
                        cudaStream_t stream) {
    int mmax, nmax;
    if (!batch_dims(batch, m, n, mmax, nmax) || !valid_opts(o)) return LLS_ERR_ARG;
    if (o.krylov != LLS_KRYLOV_CGLS || o.gemm_prec == LLS_PREC_FP32 || o.gemm_prec == LLS_PREC_FP8 || o.reorth ||
        o.panel_leaf != 0 || o.x0 != LLS_X0_ZERO)
        return LLS_ERR_UNSUPPORTED;
    if (!A || !lda || !b || !x || !ws) return LLS_ERR_ARG;
    for (int i = 0; i < batch; ++i) {
        if (!batched_supported(m[i], n[i])) return LLS_ERR_UNSUPPORTED;
        if (!A[i] || !b[i] || !x[i] || lda[i] < m[i]) return LLS_ERR_ARG;
        if (R_out && R_out[i] && (!ldr || ldr[i] < n[i])) return LLS_ERR_ARG;
    }
    if (((uintptr_t)ws & 255) != 0) return LLS_ERR_WORKSPACE;
    if (infos) memset(infos, 0, sizeof(lls_info) * (size_t)batch);
    trace_mark(stream);
    LLS_TRY(batched_upload(batch, m, n, A, lda, b, x, R_out, ldr, ws, ws_bytes, stream));
    BatchExec c;
    c.batch = batch; c.m = m; c.n = n; c.ws = ws; c.o = o; c.k = k;
    GraphKey key;
    memset(&key, 0, sizeof(key));
    key.op = 3; key.device = current_device();
    key.ints[0] = batch;
    key.ptrs[0] = ws;
    key.ws_bytes = ws_bytes; key.opts = o; key.knobs = k;
    cudaEvent_t own[3] = {nullptr, nullptr, nullptr};
    cudaEvent_t ev[3] = {nullptr, nullptr, nullptr};
    if (infos) {
        for (int i = 0; i < 3; ++i) LLS_CUDA_TRY(cudaEventCreate(&own[i]));
        for (int i = 0; i < 3; ++i) ev[i] = own[i];
    }
    int rc = run_graphed(key, stream, enqueue_batched, &c, infos ? ev : nullptr);
    trace_flush();
    if (rc != LLS_OK || !infos) {
        for (auto& e : own) if (e) cudaEventDestroy(e);
        return rc;
    }
    std::vector<double> h((size_t)16 * batch);
    LLS_CUDA_TRY(cudaMemcpyAsync(h.data(), batched_info_ptr(ws, batch, m, n), sizeof(double) * h.size(),
                                 cudaMemcpyDeviceToHost, stream));
    LLS_CUDA_TRY(cudaStreamSynchronize(stream));
    float total_ms = 0.f;
    cudaEventElapsedTime(&total_ms, ev[0], ev[1]);
    for (auto& e : own) cudaEventDestroy(e);
    int worst = LLS_OK;
    for (int i = 0; i < batch; ++i) {
        const double* d = &h[(size_t)16 * i];
        lls_info& f = infos[i];
        f.iters = (int)d[0]; f.eta = d[1]; f.fwd_est = d[2]; f.res_norm = d[3]; f.atr_norm = d[4];
        f.anorm_f = d[5]; f.xnorm = d[6]; f.a_passes = (int)d[10]; f.m_passes = (int)d[11];
        f.krylov_ms = total_ms;
        const int s = (int)d[7];
        f.status = s == 0 ? LLS_OK : (s == -2 ? LLS_ERR_SINGULAR : LLS_NOT_CONVERGED);
        if (f.status < 0) worst = f.status;
        else if (f.status > 0 && worst == LLS_OK) worst = f.status;
    }
    return worst;
}

static int batch_nmax(int batch, const int* n) {
    int mx = 0;
    for (int i = 0; n && i < batch; ++i) mx = n[i] > mx ? n[i] : mx;
    return mx;
}

static int lls_solve_batched_impl(int batch, const int* m, const int* n, const float* const* A, const int* lda,
                      const double* const* b, double* const* x, float* const* R_out, const int* ldr,
                      void* ws, size_t ws_bytes, const lls_options* opts, lls_info* infos,
                      cudaStream_t stream) {
    lls_options o;
    Knobs k;
    resolve_settings(opts, 1, batch, batch_nmax(batch, n), o, k);
    return batched_core(batch, m, n, A, lda, b, x, R_out, ldr, ws, ws_bytes, o, k, infos, stream);
}

// ---------------------------------------------------------------------------------------
// Autotuning (the paper tunes its panel by hand for its GPU, Sec. 3.1.3): timed trials of the
// implementation choices on the caller's own problem; the fastest is recorded for the shape
// and used by every later call that leaves panel_width at 0.
// ---------------------------------------------------------------------------------------
static void knobs_to_tuning(int pw, const Knobs& k, float ms, lls_tuning& t) {
    memset(&t, 0, sizeof(t));
    t.panel_width = pw;
    t.node_mode = k.node_mode;
    t.gemm_kernel = k.gemm_kernel;
    t.batched_ctas_per_sm = k.batched_ctas;
    t.krylov_ctas = k.krylov_ctas;
    t.ms = ms;
}

int lls_tuning_set(int kind, int m, int n, const lls_options* opts, const lls_tuning* t) {
    lls_options o;
    resolve(opts, o);
    if ((kind != 0 && kind != 1) || m < 1 || n < 1 || !t || !valid_opts(o)) return LLS_ERR_ARG;
    if (t->node_mode < 0 || t->node_mode > 2 || t->gemm_kernel < 0 || t->gemm_kernel > 2 ||
        t->batched_ctas_per_sm < 0 || t->krylov_ctas < 0)
        return LLS_ERR_ARG;
    if (kind == 0) {
        lls_options c = o;
        c.panel_width = t->panel_width;
        if (!valid_opts(c)) return LLS_ERR_ARG;
    }
    std::lock_guard<std::mutex> lk(g_tune_mu);
    g_tune[tune_key(kind, m, n, o)] = *t;
    return LLS_OK;
}

int lls_tuning_get(int kind, int m, int n, const lls_options* opts, lls_tuning* t) {
    lls_options o;
    resolve(opts, o);
    if ((kind != 0 && kind != 1) || !t) return LLS_ERR_ARG;
    return tuned_lookup(kind, m, n, o, *t) ? 1 : 0;
}

void lls_tuning_clear(void) {
    std::lock_guard<std::mutex> lk(g_tune_mu);
    g_tune.clear();
}

// Time of one trial: the fastest of `reps` solves after one untimed (which records the graph),
// as device time from the solve's own phase events; negative when the setting does not run.
static float trial_solve(int m, int n, const float* A, int lda, const double* b, double* x, void* ws,
                         size_t ws_bytes, const lls_options& o, const Knobs& k, int reps, cudaStream_t st) {
    if (solve_ws_bytes(m, n, o) > ws_bytes) return -1.f;
    lls_info info;
    int rc = solve_core(m, n, A, lda, b, x, nullptr, 0, ws, ws_bytes, o, k, &info, st);
    if (rc < 0) return -1.f;
    float best = -1.f;
    for (int r = 0; r < reps; ++r) {
        rc = solve_core(m, n, A, lda, b, x, nullptr, 0, ws, ws_bytes, o, k, &info, st);
        if (rc < 0) return -1.f;
        const float t = info.qr_ms + info.krylov_ms;
        if (best < 0.f || t < best) best = t;
    }
    return best;
}

size_t lls_autotune_workspace_size(int m, int n, const lls_options* opts) {
    lls_options o;
    resolve(opts, o);
    if (n < 1 || m < n || !valid_opts(o)) return 0;
    return solve_ws_bytes_auto(m, n, nullptr, o);
}

int lls_autotune(int m, int n, const float* A, int lda, const double* b, double* x, void* ws, size_t ws_bytes,
                 const lls_options* opts, int reps, lls_tuning* best, cudaStream_t stream) {
    lls_options o;
    resolve(opts, o);
    if (n < 1 || m < n || lda < m || !A || !b || !x || !ws || !best || reps < 1) return LLS_ERR_ARG;
    if (!valid_opts(o) || o.x0 == LLS_X0_GIVEN) return LLS_ERR_ARG;
    if (((uintptr_t)ws & 255) != 0) return LLS_ERR_WORKSPACE;
    // coordinate search from the defaults: panel width, then the node launches, then the
    // wide nodes' product kernel
    Knobs k = default_knobs();
    lls_options cur = o;
    cur.panel_width = 16;
    float tbest = trial_solve(m, n, A, lda, b, x, ws, ws_bytes, cur, k, reps, stream);
    for (int pw : kTuneWidths) {
        if (pw == 16) continue;
        lls_options c = o;
        c.panel_width = pw;
        if (!valid_opts(c)) continue;
        const float t = trial_solve(m, n, A, lda, b, x, ws, ws_bytes, c, k, reps, stream);
        if (t >= 0.f && (tbest < 0.f || t < tbest)) { tbest = t; cur = c; }
    }
    for (int nm = 0; nm <= 2; ++nm) {
        if (nm == k.node_mode) continue;
        Knobs c = k;
        c.node_mode = nm;
        const float t = trial_solve(m, n, A, lda, b, x, ws, ws_bytes, cur, c, reps, stream);
        if (t >= 0.f && (tbest < 0.f || t < tbest)) { tbest = t; k = c; }
    }
    for (int g = 0; g <= 2; ++g) {
        if (g == k.gemm_kernel) continue;
        Knobs c = k;
        c.gemm_kernel = g;
        const float t = trial_solve(m, n, A, lda, b, x, ws, ws_bytes, cur, c, reps, stream);
        if (t >= 0.f && (tbest < 0.f || t < tbest)) { tbest = t; k = c; }
    }
    // small problems leave most SMs idle at the size-derived Krylov grid: try wider ones
    int sms = 0, dev = 0;
    if (cudaGetDevice(&dev) == cudaSuccess) cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (sms > 0 && krylov_default_ctas(m, n) < sms) {
        const int cand[4] = {16, 64, sms, 2 * sms};
        for (int g : cand) {
            if (g <= krylov_default_ctas(m, n)) continue;
            Knobs c = k;
            c.krylov_ctas = g;
            const float t = trial_solve(m, n, A, lda, b, x, ws, ws_bytes, cur, c, reps, stream);
            if (t >= 0.f && (tbest < 0.f || t < tbest)) { tbest = t; k = c; }
        }
    }
    if (tbest < 0.f) return LLS_ERR_UNSUPPORTED;
    knobs_to_tuning(cur.panel_width, k, tbest, *best);
    return lls_tuning_set(0, m, n, &o, best);
}

int lls_autotune_batched(int batch, const int* m, const int* n, const float* const* A, const int* lda,
                         const double* const* b, double* const* x, void* ws, size_t ws_bytes,
                         const lls_options* opts, int reps, lls_tuning* best, cudaStream_t stream) {
    lls_options o;
    resolve(opts, o);
    if (!best || reps < 1) return LLS_ERR_ARG;
    // CTAs per SM, from one up to as many as fit (batched_execute caps the request)
    float tbest = -1.f;
    Knobs kb = default_knobs();
    std::vector<lls_info> infos((size_t)(batch > 0 ? batch : 1));
    for (int ctas = 1; ctas <= 4; ++ctas) {
        Knobs k = default_knobs();
        k.batched_ctas = ctas;
        int rc = batched_core(batch, m, n, A, lda, b, x, nullptr, nullptr, ws, ws_bytes, o, k, infos.data(), stream);
        if (rc < 0 && rc != LLS_NOT_CONVERGED) {
            if (ctas == 1) return rc;     // argument errors and the like: report them
            continue;
        }
        float t = -1.f;
        for (int r = 0; r < reps; ++r) {
            rc = batched_core(batch, m, n, A, lda, b, x, nullptr, nullptr, ws, ws_bytes, o, k, infos.data(), stream);
            if (rc < 0) break;
            if (t < 0.f || infos[0].krylov_ms < t) t = infos[0].krylov_ms;
        }
        if (t >= 0.f && (tbest < 0.f || t < tbest)) { tbest = t; kb = k; }
    }
    if (tbest < 0.f) return LLS_ERR_UNSUPPORTED;
    knobs_to_tuning(16, kb, tbest, *best);
    return lls_tuning_set(1, batch, batch_nmax(batch, n), &o, best);
}

// ---- entry points: LLS_DEBUG builds check the index records around each call -------------

int qr_factor(int m, int n, const float* A, int lda, float* Q, int ldq, float* R, int ldr,
              void* ws, size_t ws_bytes, const lls_options* opts, cudaStream_t stream) {
    LLS_DEBUG_BEGIN(stream);
    return debug_end(qr_factor_impl(m, n, A, lda, Q, ldq, R, ldr, ws, ws_bytes, opts, stream), stream);
}

int lls_lowp_projection(int m, int w1, int w2, int prec, const void* Q1l, const void* A2l, int ldh,
                        const int* e, float* R12, int ldr, void* R12l, int ldrl, int* f, void* ws,
                        size_t ws_bytes, cudaStream_t stream) {
    LLS_DEBUG_BEGIN(stream);
    return debug_end(lls_lowp_projection_impl(m, w1, w2, prec, Q1l, A2l, ldh, e, R12, ldr, R12l, ldrl, f, ws, ws_bytes, stream), stream);
}

int lls_lowp_update(int m, int w1, int w2, int prec, const void* Q1l, int ldh, const void* R12l,
                    int ldrl, const int* f, float* A2, int lda, void* ws, size_t ws_bytes,
                    cudaStream_t stream) {
    LLS_DEBUG_BEGIN(stream);
    return debug_end(lls_lowp_update_impl(m, w1, w2, prec, Q1l, ldh, R12l, ldrl, f, A2, lda, ws, ws_bytes, stream), stream);
}

int lls_panel_qr(int m, int b, int prec, float* W, int ldw, void* Wh, int ldh, float* R, int ldr, void* ws,
                 size_t ws_bytes, cudaStream_t stream) {
    LLS_DEBUG_BEGIN(stream);
    return debug_end(lls_panel_qr_impl(m, b, prec, W, ldw, Wh, ldh, R, ldr, ws, ws_bytes, stream), stream);
}

int lls_panel_block_qr(int m, int w1, int w2, int prec, float* W, int ldw, void* Wh, int ldh, float* R,
                       int ldr, void* ws, size_t ws_bytes, cudaStream_t stream) {
    LLS_DEBUG_BEGIN(stream);
    return debug_end(lls_panel_block_qr_impl(m, w1, w2, prec, W, ldw, Wh, ldh, R, ldr, ws, ws_bytes, stream), stream);
}

int lls_solve(int m, int n, const float* A, int lda, const double* b, double* x, float* R_out,
              int ldr, void* ws, size_t ws_bytes, const lls_options* opts, lls_info* info,
              cudaStream_t stream) {
    LLS_DEBUG_BEGIN(stream);
    const int st = debug_end(lls_solve_impl(m, n, A, lda, b, x, R_out, ldr, ws, ws_bytes, opts, info, stream), stream);
    if (st == LLS_ERR_BOUNDS && info) info->status = st;
    return st;
}

int lls_solve_host(int m, int n, const float* A, int lda, const double* b, double* x, void* ws,
                   size_t ws_bytes, const lls_options* opts, lls_info* info, cudaStream_t stream) {
    LLS_DEBUG_BEGIN(stream);
    const int st = debug_end(lls_solve_host_impl(m, n, A, lda, b, x, ws, ws_bytes, opts, info, stream), stream);
    if (st == LLS_ERR_BOUNDS && info) info->status = st;
    return st;
}

int lls_backward(int batch, const int* m, const int* n, const float* const* A, const int* lda,
                 const double* const* b, const double* const* x, const float* const* R, const int* ldr,
                 const double* const* grad_x, float* const* grad_A, const int* ldga,
                 double* const* grad_b, void* ws, size_t ws_bytes, const lls_options* opts,
                 cudaStream_t stream) {
    LLS_DEBUG_BEGIN(stream);
    return debug_end(lls_backward_impl(batch, m, n, A, lda, b, x, R, ldr, grad_x, grad_A, ldga, grad_b, ws, ws_bytes, opts, stream), stream);
}

int lls_solve_batched(int batch, const int* m, const int* n, const float* const* A, const int* lda,
                      const double* const* b, double* const* x, float* const* R_out, const int* ldr,
                      void* ws, size_t ws_bytes, const lls_options* opts, lls_info* infos,
                      cudaStream_t stream) {
    LLS_DEBUG_BEGIN(stream);
    return debug_end(lls_solve_batched_impl(batch, m, n, A, lda, b, x, R_out, ldr, ws, ws_bytes, opts, infos, stream), stream);
}

int lls_debug_build(void) { return LLS_DEBUG ? 1 : 0; }

int lls_debug_inject(int mode) {
    if (!LLS_DEBUG) return LLS_ERR_UNSUPPORTED;
    if (mode < 0 || mode > 2) return LLS_ERR_ARG;
    return panel_debug_inject(mode);
}

}  // extern "C"
