// Tall-skinny panel QR: communication-avoiding QR (Eq. caqr, Sec. 3.1.3) with CGS2 leaves.
//
// Step 1 (Eq. caqr, circled 1): the m x b panel is split into row blocks of at most
// 256 rows; each CTA factors one block in shared memory with CGS2 (classical Gram-Schmidt
// with one reorthogonalization; the paper's leaf is MGS, Alg. 4).
// Steps 2-3: the b x b R factors are stacked in groups of `fanin` and the stack is
// factored by the same routine, level by level, until one R remains. The CTA that
// finishes last in a group does that group's factorization (atomic arrival counter,
// no spin-wait), so the tree costs no extra launches.
// Steps 4-5: a second kernel multiplies each block's Q by the product of the b x b
// slices of the tree Q factors on its path to the root.
//
// Output: Q overwrites the panel in the FP32 work matrix W, a copy rounded to the
// tensor-core input type goes to Wh (feeds the next products), R goes to the R matrix.
#include "common.cuh"
#include "kernels.cuh"

namespace lls {

constexpr int kPanelThreads = 256;      // one row per thread: node height <= 256
constexpr int kPanelLd = 33;            // padded row stride of the smem block (conflict-free)

struct PanelLevels {
    int nlev;                        // tree levels above the leaves
    int nodes[kMaxPanelLevels + 1];  // node count per level (level 0 = leaves)
    int rbuf_off[kMaxPanelLevels + 1];   // first R block of each level in rbuf (units of 32x32)
    int qbuf_off[kMaxPanelLevels + 1];   // first Q block of each level in qbuf (units of 256x32)
    int cnt_off[kMaxPanelLevels + 1];    // first counter of each level
};

struct PanelArgs {
    float* W; int ldw;          // FP32 work matrix, panel at columns [c0, c0+b)
    void* Wh; int ldh;          // low-precision copy (type per `lowp`)
    float* R; int ldr;          // R output, block at [c0, c0+b)^2
    int m, c0, b, fanin, leaf_rows_unused;
    int P0;                     // number of leaf blocks
    int lowp;                   // 0 = FP16, 1 = BF16, 3 = none (FP32 products)
    float* rbuf;                // per-node R factors, 32x32 row-major blocks
    float* qbuf;                // per-node tree Q factors, 256x32 row-major blocks
    unsigned* cnt;              // per-node arrival counters (zero on entry, reset on exit)
    PanelLevels lv;
};

__device__ __forceinline__ void leaf_range(int m, int P0, int i, int& s, int& e) {
    int base = m / P0, extra = m % P0;
    s = i * base + min(i, extra);
    e = s + base + (i < extra ? 1 : 0);
}

// CGS2 of the block held in S (kPanelThreads rows x b columns, row stride kPanelLd, zero
// padded). Thread t owns row t. Column k: h = Q_<k^T a_k and a_k -= Q_<k h, twice; then
// R_<k,k = h + h', R_kk = ||a_k||, q_k = a_k / R_kk (q_k = 0 when R_kk = 0).
// On return S[:, :b] = Q and Rs (32 x 33, row-major) = R.
__device__ void cgs2_block(float* S, int b, float* red, float* Rs) {
    const int t = threadIdx.x, lane = t & 31, warp = t >> 5;
    float* myrow = S + t * kPanelLd;
    const float* wrows = S + (warp * 32) * kPanelLd;
    int parity = 0;
    for (int k = 0; k < b; ++k) {
        float hacc = 0.f;
        if (k > 0) {
            for (int pass = 0; pass < 2; ++pass) {
                // lane j: partial of q_j . a_k over this warp's 32 rows
                float part = 0.f;
#pragma unroll 8
                for (int r = 0; r < 32; ++r)
                    part = fmaf(wrows[r * kPanelLd + lane], wrows[r * kPanelLd + k], part);
                float* rb = red + parity * 256;
                parity ^= 1;
                rb[warp * 32 + lane] = part;
                __syncthreads();
                float h = 0.f;
#pragma unroll
                for (int w = 0; w < 8; ++w) h += rb[w * 32 + lane];
                if (lane >= k) h = 0.f;
                hacc += h;
                float ak = myrow[k];
                for (int j = 0; j < k; ++j) ak = fmaf(-myrow[j], __shfl_sync(kFullMask, h, j), ak);
                myrow[k] = ak;
                if (pass == 0) __syncthreads();
            }
        }
        float ak = myrow[k];
        float nn = ak * ak;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) nn += __shfl_xor_sync(kFullMask, nn, o);
        float* rb = red + parity * 256;
        parity ^= 1;
        if (lane == 0) rb[warp] = nn;
        __syncthreads();
        float tot = 0.f;
#pragma unroll
        for (int w = 0; w < 8; ++w) tot += rb[w];
        float nrm = sqrtf(tot);
        myrow[k] = nrm > 0.f ? ak / nrm : 0.f;
        if (warp == 0 && lane < k) Rs[lane * kPanelLd + k] = hacc;
        if (t == 0) Rs[k * kPanelLd + k] = nrm;
        __syncthreads();
    }
}

__global__ void __launch_bounds__(kPanelThreads)
panel_leaf_tree_kernel(PanelArgs a) {
    __shared__ float S[kPanelThreads * kPanelLd];
    __shared__ float red[2 * 256];
    __shared__ float Rs[32 * kPanelLd];
    __shared__ int s_last;
    const int t = threadIdx.x;
    const int b = a.b;

    for (int i = t; i < 32 * kPanelLd; i += kPanelThreads) Rs[i] = 0.f;

    // ---- step 1: factor this CTA's row block ----
    int s, e;
    leaf_range(a.m, a.P0, blockIdx.x, s, e);
    const int rows = e - s;
    float* myrow = S + t * kPanelLd;
    for (int j = 0; j < 32; ++j) {
        float v = 0.f;
        if (t < rows && j < b) v = a.W[(size_t)(s + t) + (size_t)(a.c0 + j) * a.ldw];
        myrow[j] = v;
    }
    __syncthreads();
    cgs2_block(S, b, red, Rs);
    if (t < rows)
        for (int j = 0; j < b; ++j) a.W[(size_t)(s + t) + (size_t)(a.c0 + j) * a.ldw] = myrow[j];

    if (a.P0 == 1) {   // the leaf is the whole panel: R11 is final
        for (int i = t; i < b * b; i += kPanelThreads) {
            int r = i % b, c = i / b;
            a.R[(size_t)(a.c0 + r) + (size_t)(a.c0 + c) * a.ldr] = r <= c ? Rs[r * kPanelLd + c] : 0.f;
        }
        return;
    }
    {
        float* dst = a.rbuf + (size_t)(a.lv.rbuf_off[0] + blockIdx.x) * 1024;
        for (int i = t; i < 1024; i += kPanelThreads) dst[i] = Rs[(i >> 5) * kPanelLd + (i & 31)];
    }

    // ---- steps 2-3: combine stacked R factors up the tree (last arriver does the work) ----
    int node = blockIdx.x;
    for (int l = 0; l < a.lv.nlev; ++l) {
        const int parent = node / a.fanin;
        const int nch = min(a.fanin, a.lv.nodes[l] - parent * a.fanin);
        __threadfence();
        __syncthreads();
        if (t == 0) {
            unsigned* c = a.cnt + a.lv.cnt_off[l + 1] + parent;
            unsigned old = atomicAdd(c, 1u);
            s_last = (old == (unsigned)(nch - 1));
            if (s_last) atomicExch(c, 0u);   // self-reset for the next panel
        }
        __syncthreads();
        if (!s_last) return;
        __threadfence();
        // stack the children's R factors: row t = child (t / b), row (t % b) of its R
        const int child = t / b, rr = t % b;
        const float* src = a.rbuf + (size_t)(a.lv.rbuf_off[l] + parent * a.fanin + child) * 1024;
        for (int j = 0; j < 32; ++j) {
            float v = 0.f;
            if (child < nch && j < b) v = __ldcg(src + rr * 32 + j);
            myrow[j] = v;
        }
        for (int i = t; i < 32 * kPanelLd; i += kPanelThreads) Rs[i] = 0.f;
        __syncthreads();
        cgs2_block(S, b, red, Rs);
        // tree Q of this node (rows = nch*b, row-major 256 x 32 block)
        float* qdst = a.qbuf + (size_t)(a.lv.qbuf_off[l + 1] + parent) * (256 * 32);
        for (int j = 0; j < 32; ++j) qdst[t * 32 + j] = myrow[j];
        if (a.lv.nodes[l + 1] == 1) {
            for (int i = t; i < b * b; i += kPanelThreads) {
                int r = i % b, c = i / b;
                a.R[(size_t)(a.c0 + r) + (size_t)(a.c0 + c) * a.ldr] = r <= c ? Rs[r * kPanelLd + c] : 0.f;
            }
            return;
        }
        float* dst = a.rbuf + (size_t)(a.lv.rbuf_off[l + 1] + parent) * 1024;
        for (int i = t; i < 1024; i += kPanelThreads) dst[i] = Rs[(i >> 5) * kPanelLd + (i & 31)];
        node = parent;
    }
}

template <typename TL>
__device__ __forceinline__ void store_lowp(void* Wh, size_t idx, float v) {
    reinterpret_cast<TL*>(Wh)[idx] = LowPrec<TL>::from_float(v);
}

// Steps 4-5: Q_i <- Q_i * (S_1 S_2 ... S_top), S_l the b x b slice of the level-l tree Q on
// the block's path; writes the FP32 Q and its low-precision copy.
__global__ void __launch_bounds__(kPanelThreads)
panel_reconstruct_kernel(PanelArgs a) {
    __shared__ float T[32 * 33];
    __shared__ float U[32 * 33];
    const int t = threadIdx.x;
    const int b = a.b;
    // T = I
    for (int i = t; i < 32 * 33; i += kPanelThreads) T[i] = 0.f;
    __syncthreads();
    if (t < 32) T[t * 33 + t] = 1.f;
    __syncthreads();
    int node = blockIdx.x;
    for (int l = 0; l < a.lv.nlev; ++l) {
        const int parent = node / a.fanin, child = node % a.fanin;
        const float* q = a.qbuf + (size_t)(a.lv.qbuf_off[l + 1] + parent) * (256 * 32) + (size_t)child * b * 32;
        // U = T * S_l (b x b), S_l[r][c] = q[r*32 + c]
        for (int i = t; i < b * b; i += kPanelThreads) {
            int r = i / b, c = i % b;
            float acc = 0.f;
            for (int k = 0; k < b; ++k) acc = fmaf(T[r * 33 + k], __ldcg(q + k * 32 + c), acc);
            U[r * 33 + c] = acc;
        }
        __syncthreads();
        for (int i = t; i < b * b; i += kPanelThreads) {
            int r = i / b, c = i % b;
            T[r * 33 + c] = U[r * 33 + c];
        }
        __syncthreads();
        node = parent;
    }
    int s, e;
    leaf_range(a.m, a.P0, blockIdx.x, s, e);
    if (t >= e - s) return;
    const size_t row = (size_t)(s + t);
    float q[32];
#pragma unroll
    for (int j = 0; j < 32; ++j) q[j] = j < b ? a.W[row + (size_t)(a.c0 + j) * a.ldw] : 0.f;
    for (int j = 0; j < b; ++j) {
        float acc = 0.f;
#pragma unroll
        for (int k = 0; k < 32; ++k) acc = fmaf(q[k], T[k * 33 + j], acc);
        const size_t widx = row + (size_t)(a.c0 + j) * a.ldw;
        a.W[widx] = acc;
        const size_t hidx = row + (size_t)(a.c0 + j) * a.ldh;
        if (a.lowp == 0) store_lowp<__half>(a.Wh, hidx, acc);
        else if (a.lowp == 1) store_lowp<__nv_bfloat16>(a.Wh, hidx, acc);
    }
}

// ---------------------------------------------------------------------------------------
// Host side
// ---------------------------------------------------------------------------------------
static void panel_levels(int m, int b, PanelLevels& lv, int& P0, int& fanin) {
    P0 = ceil_div(m, kPanelThreads);
    int bp = b <= 8 ? 8 : (b <= 16 ? 16 : 32);
    fanin = kPanelThreads / bp;
    lv.nodes[0] = P0;
    lv.nlev = 0;
    while (lv.nodes[lv.nlev] > 1) {
        lv.nodes[lv.nlev + 1] = ceil_div(lv.nodes[lv.nlev], fanin);
        lv.nlev++;
    }
    int ro = 0, qo = 0, co = 0;
    for (int l = 0; l <= lv.nlev; ++l) {
        lv.rbuf_off[l] = ro;
        ro += lv.nodes[l];
        lv.qbuf_off[l] = qo;
        lv.cnt_off[l] = co;
        if (l > 0) { qo += lv.nodes[l]; co += lv.nodes[l]; }
    }
}

void panel_scratch_sizes(int m, size_t& rbuf_floats, size_t& qbuf_floats, size_t& cnt_words) {
    PanelLevels lv;
    int P0, fanin;
    panel_levels(m, 32, lv, P0, fanin);   // widest panel has the smallest fan-in, so the most nodes
    size_t nodes = 0, upper = 0;
    for (int l = 0; l <= lv.nlev; ++l) { nodes += lv.nodes[l]; if (l > 0) upper += lv.nodes[l]; }
    rbuf_floats = nodes * 1024;
    qbuf_floats = (upper + 1) * 256 * 32;
    cnt_words = upper + 1;
}

int panel_qr(const PanelCall& c, cudaStream_t st) {
    PanelArgs a;
    a.W = c.W; a.ldw = c.ldw; a.Wh = c.Wh; a.ldh = c.ldh; a.R = c.R; a.ldr = c.ldr;
    a.m = c.m; a.c0 = c.c0; a.b = c.b; a.lowp = c.lowp;
    a.rbuf = c.rbuf; a.qbuf = c.qbuf; a.cnt = c.cnt; a.leaf_rows_unused = 0;
    panel_levels(c.m, c.b, a.lv, a.P0, a.fanin);
    if (a.lv.nlev > kMaxPanelLevels || c.b < 1 || c.b > 32) return LLS_ERR_UNSUPPORTED;
    panel_leaf_tree_kernel<<<a.P0, kPanelThreads, 0, st>>>(a);
    LLS_LAUNCH_CHECK();
    panel_reconstruct_kernel<<<a.P0, kPanelThreads, 0, st>>>(a);
    LLS_LAUNCH_CHECK();
    return LLS_OK;
}

}  // namespace lls
