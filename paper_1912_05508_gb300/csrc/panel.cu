// Tall-skinny panel QR: communication-avoiding QR (Eq. caqr, Sec. 3.1.3) with CGS2 leaves.
//
// Step 1 (Eq. caqr, circled 1): the m x b panel is split into row blocks of at most 1024 rows;
// each CTA factors one block with CGS2 (classical Gram-Schmidt with one reorthogonalization;
// the paper's leaf is MGS, Alg. 4), holding the block in registers, 4 rows per thread.
// Steps 2-3: the b x b R factors are stacked in groups of `fanin` (1024 / b rows) and the
// stack is factored by the same routine, level by level, until one R remains. The CTA that
// finishes last in a group does that group's factorization (atomic arrival counter, no
// spin-wait), so the tree costs no extra launches.
// Steps 4-5: a second kernel multiplies each block's Q by the product of the b x b slices
// of the tree Q factors on its path to the root (skipped when the panel is one block).
//
// CGS2 column k, all in registers: one block-wide reduction gives h = Q_<k^T a_k, then
// a_k -= Q_<k h; a second gives h' = Q_<k^T a_k together with ||a_k||^2, then a_k -= Q_<k h'
// and ||a_k''||^2 = ||a_k||^2 - ||h'||^2 (h' is at the rounding level after the first pass;
// when it is not, the norm is reduced directly). R_<k,k = h + h', R_kk = ||a_k''||,
// q_k = a_k'' / R_kk (q_k = 0 when R_kk = 0). Each reduction is a butterfly transpose-
// reduction across the warp followed by one pass through shared memory.
//
// Output: Q overwrites the panel in the FP32 work matrix W, a copy rounded to the
// tensor-core input type goes to Wh (feeds the next products), R goes to the R matrix.
#include "cgs2.cuh"
#include "common.cuh"
#include "kernels.cuh"

namespace lls {

struct PanelLevels {
    int nlev;                              // tree levels above the leaves
    int nodes[kMaxPanelLevels + 1];        // node count per level (level 0 = leaves)
    int rbuf_off[kMaxPanelLevels + 1];     // first R block of each level in rbuf (32x32 blocks)
    int qbuf_off[kMaxPanelLevels + 1];     // first Q block of each level in qbuf (1024x32 blocks)
    int cnt_off[kMaxPanelLevels + 1];      // first counter of each level
};

struct PanelArgs {
    float* W; int ldw;
    void* Wh; int ldh;
    float* R; int ldr;
    int m, c0, b, fanin, P0, lowp;
    float* rbuf;
    float* qbuf;
    unsigned* cnt;      // per-node arrival counters (zero on entry, self-resetting)
    unsigned* sync;     // [0] root-done flag, [1] exit count (one-launch path)
    int* err;
    PanelLevels lv;
};

__device__ __forceinline__ void leaf_range(int m, int P0, int i, int& s, int& e) {
    const int base = m / P0, extra = m % P0;
    s = i * base + min(i, extra);
    e = s + base + (i < extra ? 1 : 0);
}

template <typename TL>
__device__ __forceinline__ void store_lowp(void* Wh, size_t idx, float v) {
    reinterpret_cast<TL*>(Wh)[idx] = LowPrec<TL>::from_float(v);
}

__device__ __forceinline__ void store_q(const PanelArgs& a, int row, int j, float q) {
    a.W[(size_t)row + (size_t)(a.c0 + j) * a.ldw] = q;
    const size_t hidx = (size_t)row + (size_t)(a.c0 + j) * a.ldh;
    if (a.lowp == 0) store_lowp<__half>(a.Wh, hidx, q);
    else if (a.lowp == 1) store_lowp<__nv_bfloat16>(a.Wh, hidx, q);
}

__device__ __forceinline__ void write_r11(const PanelArgs& a, const float* Rs) {
    for (int i = threadIdx.x; i < a.b * a.b; i += kPanelThreads) {
        const int r = i % a.b, c = i / a.b;
        a.R[(size_t)(a.c0 + r) + (size_t)(a.c0 + c) * a.ldr] = r <= c ? Rs[r * 33 + c] : 0.f;
    }
}

__device__ __forceinline__ void write_rblock(float* dst, const float* Rs) {
    for (int i = threadIdx.x; i < 1024; i += kPanelThreads) dst[i] = Rs[(i >> 5) * 33 + (i & 31)];
}

// Load the CTA's leaf block (rows t + 256 r of [s, s + rows)) and factor it.
template <int B>
__device__ __forceinline__ void leaf_factor(const PanelArgs& a, float (&v)[kRPT][B], float* red, float* Rs,
                                            int s, int rows) {
    const int t = threadIdx.x, b = a.b;
#pragma unroll
    for (int r = 0; r < kRPT; ++r) {
        const int lr = t + r * kPanelThreads;
#pragma unroll
        for (int j = 0; j < B; ++j)
            v[r][j] = (lr < rows && j < b) ? a.W[(size_t)(s + lr) + (size_t)(a.c0 + j) * a.ldw] : 0.f;
    }
    __syncthreads();
    cgs2_block<B>(v, b, red, Rs);
}

// Store the factored block's Q (q_j at register position B - b + j): to W and Wh when
// `final`, to W only otherwise.
template <int B>
__device__ __forceinline__ void store_leaf_q(const PanelArgs& a, const float (&v)[kRPT][B], int s, int rows,
                                             bool final) {
    const int t = threadIdx.x, off = B - a.b;
#pragma unroll
    for (int r = 0; r < kRPT; ++r) {
        const int lr = t + r * kPanelThreads;
        if (lr >= rows) continue;
#pragma unroll
        for (int p = 0; p < B; ++p) {
            const int j = p - off;
            if (j < 0) continue;
            if (final) store_q(a, s + lr, j, v[r][p]);
            else a.W[(size_t)(s + lr) + (size_t)(a.c0 + j) * a.ldw] = v[r][p];
        }
    }
}

// Steps 2-3: climb the tree from leaf `node`; at each level the CTA that arrives last in its
// group factors the group's stacked R factors. Returns true for the CTA that factored the
// root (R11 written), false for a CTA that stopped because it was not last.
template <int B>
__device__ bool climb_tree(const PanelArgs& a, float (&v)[kRPT][B], float* red, float* Rs, int node,
                           int* s_last) {
    const int t = threadIdx.x, b = a.b, off = B - b;
    for (int l = 0; l < a.lv.nlev; ++l) {
        const int parent = node / a.fanin;
        const int nch = min(a.fanin, a.lv.nodes[l] - parent * a.fanin);
        __threadfence();
        __syncthreads();
        if (t == 0) {
            unsigned* c = a.cnt + a.lv.cnt_off[l + 1] + parent;
            const unsigned old = atomicAdd(c, 1u);
            *s_last = (old == (unsigned)(nch - 1));
            if (*s_last) atomicExch(c, 0u);   // self-reset for the next panel
        }
        __syncthreads();
        if (!*s_last) return false;
        __threadfence();
        const float* src0 = a.rbuf + (size_t)(a.lv.rbuf_off[l] + parent * a.fanin) * 1024;
#pragma unroll
        for (int r = 0; r < kRPT; ++r) {
            const int rho = t + r * kPanelThreads;        // stacked row
            const int child = rho / b, rr = rho % b;
#pragma unroll
            for (int j = 0; j < B; ++j)
                v[r][j] = (child < nch && j < b) ? __ldcg(src0 + (size_t)child * 1024 + rr * 32 + j) : 0.f;
        }
        for (int i = t; i < 32 * 33; i += kPanelThreads) Rs[i] = 0.f;
        __syncthreads();
        cgs2_block<B>(v, b, red, Rs);
        float* qdst = a.qbuf + (size_t)(a.lv.qbuf_off[l + 1] + parent) * (kNodeRows * 32);
#pragma unroll
        for (int r = 0; r < kRPT; ++r) {
            const int rho = t + r * kPanelThreads;
            if (rho < nch * b)
#pragma unroll
                for (int p = 0; p < B; ++p)
                    if (p >= off) qdst[rho * 32 + (p - off)] = v[r][p];
        }
        if (a.lv.nodes[l + 1] == 1) {
            write_r11(a, Rs);
            return true;
        }
        write_rblock(a.rbuf + (size_t)(a.lv.rbuf_off[l + 1] + parent) * 1024, Rs);
        node = parent;
    }
    return false;
}

// Steps 4-5 for leaf block `leaf`: Q_i <- Q_i (S_1 S_2 ... S_top), S_l the b x b slice of the
// level-l tree Q on the block's path; reads the leaf Q from W, writes Q to W and Wh.
template <int B>
__device__ void reconstruct(const PanelArgs& a, int leaf, float* T, float* U) {
    const int t = threadIdx.x, b = a.b;
    for (int i = t; i < 32 * 33; i += kPanelThreads) T[i] = (i / 33 == i % 33) ? 1.f : 0.f;
    __syncthreads();
    int node = leaf;
    for (int l = 0; l < a.lv.nlev; ++l) {
        const int parent = node / a.fanin, child = node % a.fanin;
        const float* q = a.qbuf + (size_t)(a.lv.qbuf_off[l + 1] + parent) * (kNodeRows * 32) + (size_t)child * b * 32;
        for (int i = t; i < b * b; i += kPanelThreads) {
            const int r = i / b, c = i % b;
            float acc = 0.f;
            for (int k = 0; k < b; ++k) acc = fmaf(T[r * 33 + k], __ldcg(q + k * 32 + c), acc);
            U[r * 33 + c] = acc;
        }
        __syncthreads();
        for (int i = t; i < b * b; i += kPanelThreads) T[(i / b) * 33 + (i % b)] = U[(i / b) * 33 + (i % b)];
        __syncthreads();
        node = parent;
    }
    int s, e;
    leaf_range(a.m, a.P0, leaf, s, e);
    const int rows = e - s;
#pragma unroll 1
    for (int r = 0; r < kRPT; ++r) {
        const int lr = t + r * kPanelThreads;
        if (lr >= rows) break;
        const size_t row = (size_t)(s + lr);
        float q[B];
#pragma unroll
        for (int j = 0; j < B; ++j) q[j] = j < b ? __ldcg(a.W + row + (size_t)(a.c0 + j) * a.ldw) : 0.f;
#pragma unroll
        for (int j = 0; j < B; ++j) {
            if (j >= b) break;
            float acc = 0.f;
#pragma unroll
            for (int k = 0; k < B; ++k) acc = fmaf(q[k], T[k * 33 + j], acc);
            store_q(a, (int)row, j, acc);
        }
    }
}

// Two-launch path, step 1-3 (any number of leaf blocks).
template <int B>
__global__ void __launch_bounds__(kPanelThreads, 1)
panel_leaf_tree_kernel(PanelArgs a) {
    __shared__ float red[kRedFloats];
    __shared__ float Rs[32 * 33];
    __shared__ int s_last;
    for (int i = threadIdx.x; i < 32 * 33; i += kPanelThreads) Rs[i] = 0.f;
    int s, e;
    leaf_range(a.m, a.P0, blockIdx.x, s, e);
    float v[kRPT][B];
    leaf_factor<B>(a, v, red, Rs, s, e - s);
    if (a.P0 == 1) {   // the block is the whole panel: Q and R are final
        store_leaf_q<B>(a, v, s, e - s, true);
        write_r11(a, Rs);
        return;
    }
    store_leaf_q<B>(a, v, s, e - s, false);
    write_rblock(a.rbuf + (size_t)(a.lv.rbuf_off[0] + blockIdx.x) * 1024, Rs);
    climb_tree<B>(a, v, red, Rs, blockIdx.x, &s_last);
}

// Two-launch path, steps 4-5.
template <int B>
__global__ void __launch_bounds__(kPanelThreads)
panel_reconstruct_kernel(PanelArgs a) {
    __shared__ float T[32 * 33];
    __shared__ float U[32 * 33];
    reconstruct<B>(a, blockIdx.x, T, U);
}

// One-launch path (cooperative launch, all leaf CTAs resident): after the tree, every CTA
// waits (bounded) for the root CTA's completion flag, then rebuilds its own block. The last
// CTA to finish resets the flag words for the next panel.
template <int B>
__global__ void __launch_bounds__(kPanelThreads, 1)
panel_coop_kernel(PanelArgs a) {
    __shared__ float red[kRedFloats];
    __shared__ float Rs[32 * 33];
    __shared__ float U[32 * 33];
    __shared__ int s_last, s_ok;
    for (int i = threadIdx.x; i < 32 * 33; i += kPanelThreads) Rs[i] = 0.f;
    int s, e;
    leaf_range(a.m, a.P0, blockIdx.x, s, e);
    {
        float v[kRPT][B];
        leaf_factor<B>(a, v, red, Rs, s, e - s);
        store_leaf_q<B>(a, v, s, e - s, false);
        write_rblock(a.rbuf + (size_t)(a.lv.rbuf_off[0] + blockIdx.x) * 1024, Rs);
        const bool root = climb_tree<B>(a, v, red, Rs, blockIdx.x, &s_last);
        if (root) {
            __threadfence();
            __syncthreads();
            if (threadIdx.x == 0) atomicExch(a.sync, 1u);
        }
    }
    if (threadIdx.x == 0) {
        int ok = 1;
        const unsigned long long t0 = globaltimer_ns();
        while (atomicAdd(a.sync, 0u) == 0u) {
            if (globaltimer_ns() - t0 > kSpinLimitNs) {
                atomicCAS(a.err, DEV_OK, DEV_TIMEOUT);
                ok = 0;
                break;
            }
            __nanosleep(200);
        }
        __threadfence();
        s_ok = ok;
    }
    __syncthreads();
    if (s_ok) reconstruct<B>(a, blockIdx.x, Rs, U);
    __syncthreads();
    if (threadIdx.x == 0) {
        __threadfence();
        if (atomicAdd(a.sync + 1, 1u) == (unsigned)(a.P0 - 1)) {
            atomicExch(a.sync + 1, 0u);
            atomicExch(a.sync, 0u);
        }
    }
}

// ---------------------------------------------------------------------------------------
// Host side
// ---------------------------------------------------------------------------------------
static int bucket(int b) { return b <= 8 ? 8 : (b <= 16 ? 16 : 32); }

constexpr int kSyncWords = 2 + kFlatBarWords;   // cnt[0..1]: root-done flag and exit count of the
                                                  // one-launch path; then the one-level panel's barrier

static void panel_levels(int m, int b, PanelLevels& lv, int& P0, int& fanin) {
    P0 = ceil_div(m, kNodeRows);
    fanin = kNodeRows / bucket(b);
    lv.nodes[0] = P0;
    lv.nlev = 0;
    while (lv.nodes[lv.nlev] > 1 && lv.nlev < kMaxPanelLevels) {
        lv.nodes[lv.nlev + 1] = ceil_div(lv.nodes[lv.nlev], fanin);
        lv.nlev++;
    }
    int ro = 0, qo = 0, co = kSyncWords;
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
    qbuf_floats = (upper + 1) * (size_t)kNodeRows * 32;
    cnt_words = upper + kSyncWords + 1;
}

template <int B>
static int coop_capacity() {
    static int cap = -1;
    if (cap < 0) {
        int dev = 0, sms = 0, per = 0;
        if (cudaGetDevice(&dev) != cudaSuccess ||
            cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess ||
            cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, panel_coop_kernel<B>, kPanelThreads, 0) != cudaSuccess)
            cap = 0;
        else
            cap = sms * per;
    }
    return cap;
}

template <int B>
static int launch_panel(PanelArgs& a, cudaStream_t st) {
    if (a.P0 > 1 && a.P0 <= coop_capacity<B>()) {
        void* args[] = {&a};
        LLS_CUDA_TRY(cudaLaunchCooperativeKernel((void*)panel_coop_kernel<B>, dim3(a.P0), dim3(kPanelThreads), args, 0, st));
        LLS_LAUNCH_CHECK("panel_coop", st);
        return LLS_OK;
    }
    panel_leaf_tree_kernel<B><<<a.P0, kPanelThreads, 0, st>>>(a);
    LLS_LAUNCH_CHECK("panel_leaf_tree", st);
    if (a.P0 > 1) {
        panel_reconstruct_kernel<B><<<a.P0, kPanelThreads, 0, st>>>(a);
        LLS_LAUNCH_CHECK("panel_reconstruct", st);
    }
    return LLS_OK;
}

int panel_qr(const PanelCall& c, cudaStream_t st) {
    if (c.b < 1 || c.b > 32) return LLS_ERR_UNSUPPORTED;
    // one-level tree when the stacked leaf R factors fit one block (panel_flat.cu)
    const int flat = panel_flat_qr(c, st);
    if (flat != LLS_ERR_UNSUPPORTED || c.leaf != 0) return flat;   // MGS leaves: one-level panels only
    PanelArgs a;
    a.W = c.W; a.ldw = c.ldw; a.Wh = c.Wh; a.ldh = c.ldh; a.R = c.R; a.ldr = c.ldr;
    a.m = c.m; a.c0 = c.c0; a.b = c.b; a.lowp = c.lowp;
    a.rbuf = c.rbuf; a.qbuf = c.qbuf; a.cnt = c.cnt; a.sync = c.cnt; a.err = c.err;
    panel_levels(c.m, c.b, a.lv, a.P0, a.fanin);
    if (a.lv.nodes[a.lv.nlev] != 1) return LLS_ERR_UNSUPPORTED;
    const int bk = bucket(c.b);
    if (bk == 8) return launch_panel<8>(a, st);
    if (bk == 16) return launch_panel<16>(a, st);
    return launch_panel<32>(a, st);
}

}  // namespace lls
