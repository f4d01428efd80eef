// One narrow recursion node (the projection and update of Alg. 2, w1 <= 32 columns) in a single cooperative
// launch, with the same rounding points as the tensor-core path:
//
//   A. every CTA owns 256 rows: it loads its rows of Q1 (product precision) and A2 (FP32)
//      and forms the column maxima of |A2| over those rows;
//   B. e_j from the CTA's maxima (FP16: max * 2^e_j in [2^14, 2^15); BF16: e_j = 0), the
//      CTA's rows of A2 rounded as round(A2 * 2^e_j), and the CTA's partial Q1l^T A2l by
//      warp-level FP16/BF16 products with FP32 accumulation, times 2^-e_j; -> grid barrier
//   C. CTA j sums column j of the partials in a fixed order into R12 (to R), f_j from
//      max |R12_:j|, R12l = round(R12 * 2^f_j);                            -> grid barrier
//   D. every CTA updates its rows: A2 -= (Q1l R12l) * 2^-f_j, in FP32.
//
// At narrow nodes the four separate kernels of the wide-node path (cast, projection,
// split-K reduce, update) each cost a launch and a pass through L2 for a few MB of data; here
// the rows stay on chip from A to D. Results equal the wide-node path's up to the order of
// the FP32 accumulation: the wide-node path scales column j by the exponent of its maximum
// over all rows, each CTA here by the exponent of its own rows' maximum (never smaller).
// Power-of-two scaling commutes with rounding to FP16 and with the FP32 accumulation while
// the values stay normal, so each partial times 2^-e_j is the same number either way, and
// no grid barrier is needed to agree on the exponents. Every grid-barrier wait is bounded.
#include <mma.h>

#include "cgs2.cuh"
#include "common.cuh"
#include "kernels.cuh"

namespace lls {
namespace {

using namespace nvcuda;

constexpr int kNT = 256;                 // threads per CTA = rows per CTA
constexpr int kNW = kNT / 32;
constexpr int kLdK = kNT + 8;            // halves per column of the K-contiguous tiles
constexpr int kNodeMaxW1 = 32;           // widest left half handled here (at w1 = 64 the
                                         // tensor-core path measured as fast)

struct NodeArgs {
    float* W; int ldw;                   // FP32 work matrix: Q1 columns [c0, c0+w1), A2 after
    const void* Wh; int ldh;             // product-precision copy (Q1l)
    int m, c0, w1, w2, kind;             // kind: 1 FP16 scaling, 0 none (BF16)
    float* R; int ldr;                   // R12 block goes to R[c0 .. c0+w1, c0+w1 .. c0+w)
    float* part;                         // gridDim.x partial planes of W1 x W1 (column-major)
    void* R12l;                          // W1 x W1 scaled low-precision R12 (column-major)
    int* f;                              // w2 exponents of R12's columns
    unsigned* bar;                       // grid barrier words (count, generation)
    int* err;
};

template <typename TL, int W1>
struct NodeSmem {
    __align__(32) TL Qs[W1][kLdK];       // Q1l^T rows: Qs[i][r]      (projection operand A)
    __align__(32) TL As[W1][kLdK];       // scaled A2l: As[j][r]      (projection operand B)
    __align__(32) TL QsT[kNT][W1 + 8];   // Q1l rows: QsT[r][i]       (update operand A)
    __align__(32) TL Rl[W1][W1];         // R12l column-major         (update operand B)
    __align__(32) float Us[kNT][W1 + 4]; // update products, row-major
    float red[2][kNW][32];               // column maxima, up to two chunks of 32 columns
    float sc[W1];                        // 2^e_j (phase B), 2^-f_j (phase D)
    float einv[W1];                      // 2^-e_j (phase B)
    float part_g[kNT];
};

template <typename TL> struct WmmaT;
template <> struct WmmaT<__half> { using type = __half; };
template <> struct WmmaT<__nv_bfloat16> { using type = __nv_bfloat16; };

template <typename TL, int W1>
__global__ void __launch_bounds__(kNT) node_fused_kernel(NodeArgs a) {
    extern __shared__ __align__(128) unsigned char node_smem[];
    NodeSmem<TL, W1>& sm = *reinterpret_cast<NodeSmem<TL, W1>*>(node_smem);
    const int t = threadIdx.x, lane = t & 31, warp = t >> 5;
    const int row = blockIdx.x * kNT + t;
    const bool valid = row < a.m;
    const int w1 = a.w1, w2 = a.w2, cA = a.c0 + w1;
    const TL* Wh = reinterpret_cast<const TL*>(a.Wh);
    const TL zero = LowPrec<TL>::from_float(0.f);

    // ---- A: load this CTA's rows; column maxima of |A2| ------------------------------------
    float av[W1];
#pragma unroll
    for (int j = 0; j < W1; ++j)
        av[j] = (valid && j < w2 && LLS_INB(row < a.ldw)) ? a.W[(size_t)row + (size_t)(cA + j) * a.ldw] : 0.f;
#pragma unroll
    for (int i = 0; i < W1; ++i) {
        const TL q = (valid && i < w1 && LLS_INB(row < a.ldh)) ? Wh[(size_t)row + (size_t)(a.c0 + i) * a.ldh] : zero;
        sm.Qs[i][t] = q;
        sm.QsT[t][i] = q;
    }
    if (a.kind != 0) {
        // per chunk of (up to) 32 columns: lane L ends with the warp maximum of column 32 c + L
        constexpr int kCh = W1 < 32 ? W1 : 32;
#pragma unroll
        for (int c = 0; c < W1 / kCh; ++c) {
            float mx[kCh];
#pragma unroll
            for (int j = 0; j < kCh; ++j) mx[j] = fabsf(av[c * kCh + j]);
            sm.red[c][warp][lane] = warp_transpose_max<kCh>(mx);
        }
        __syncthreads();
        if (t < W1) {
            float m = 0.f;
#pragma unroll
            for (int q = 0; q < kNW; ++q) m = fmaxf(m, sm.red[t / kCh][q][t % kCh]);
            const int e = scale_exponent(a.kind, t < w2 ? m : 0.f);
            sm.sc[t] = pow2f(e);
            sm.einv[t] = pow2f(-e);
        }
    } else if (t < W1) {
        sm.sc[t] = 1.f;
        sm.einv[t] = 1.f;
    }
    __syncthreads();

    // ---- B: scaled low-precision A2 rows, partial Q1l^T A2l -------------------------------
#pragma unroll
    for (int j = 0; j < W1; ++j) sm.As[j][t] = LowPrec<TL>::from_float(av[j] * sm.sc[j]);
    __syncthreads();
    using WT = typename WmmaT<TL>::type;
    constexpr int kTiles = (W1 / 16) * (W1 / 16);
    for (int tile = warp; tile < kTiles; tile += kNW) {
        const int mt = tile / (W1 / 16), nt = tile % (W1 / 16);
        wmma::fragment<wmma::accumulator, 16, 16, 16, float> acc;
        wmma::fill_fragment(acc, 0.f);
#pragma unroll 4
        for (int k0 = 0; k0 < kNT; k0 += 16) {
            wmma::fragment<wmma::matrix_a, 16, 16, 16, WT, wmma::row_major> fa;
            wmma::fragment<wmma::matrix_b, 16, 16, 16, WT, wmma::col_major> fb;
            wmma::load_matrix_sync(fa, reinterpret_cast<const WT*>(&sm.Qs[mt * 16][k0]), kLdK);
            wmma::load_matrix_sync(fb, reinterpret_cast<const WT*>(&sm.As[nt * 16][k0]), kLdK);
            wmma::mma_sync(acc, fa, fb, acc);
        }
        // the tile through shared memory (Us is free until phase D), unscaled by 2^-e_j (exact)
        float* us = &sm.Us[0][0] + tile * 256;
        wmma::store_matrix_sync(us, acc, 16, wmma::mem_col_major);
        __syncwarp();
        float* pp = a.part + (size_t)blockIdx.x * (W1 * W1) + (size_t)(nt * 16) * W1 + mt * 16;   // plane of W1 x W1
        for (int e = lane; e < 256; e += 32) {
            const int i = e & 15, j = e >> 4;
            pp[(size_t)j * W1 + i] = us[e] * sm.einv[nt * 16 + j];
        }
    }
    if (!grid_barrier(a.bar, gridDim.x, a.err)) return;

    // ---- C: fixed-order sum of the partials, R12 and its scaled low-precision copy --------
    for (int j = blockIdx.x; j < W1; j += gridDim.x) {
        if (j >= w2) {                            // padding columns of R12l
            if (t < W1) reinterpret_cast<TL*>(a.R12l)[(size_t)t + (size_t)j * W1] = zero;
            continue;
        }
        constexpr int G = kNT / W1;               // split groups
        const int i0 = t % W1, g = t / W1;
        const int P = gridDim.x;
        float s = 0.f;
        const float* p = a.part + (size_t)i0 + (size_t)j * W1;
        int z = g;
        for (; z + 3 * G < P; z += 4 * G) {
            const float x0 = __ldcg(p + (size_t)z * (W1 * W1)), x1 = __ldcg(p + (size_t)(z + G) * (W1 * W1));
            const float x2 = __ldcg(p + (size_t)(z + 2 * G) * (W1 * W1));
            const float x3 = __ldcg(p + (size_t)(z + 3 * G) * (W1 * W1));
            s += x0; s += x1; s += x2; s += x3;
        }
        for (; z < P; z += G) s += __ldcg(p + (size_t)z * (W1 * W1));
        __syncthreads();                          // part_g and sc[0] of the previous column are consumed
        sm.part_g[t] = s;
        __syncthreads();
        float r12 = 0.f;
        if (t < W1) {
            float tot = 0.f;
#pragma unroll
            for (int q = 0; q < G; ++q) tot += sm.part_g[q * W1 + t];
            r12 = tot;
            if (t < w1 && LLS_INB(a.c0 + t < a.ldr)) a.R[(size_t)(a.c0 + t) + (size_t)(cA + j) * a.ldr] = r12;
        }
        float mx = (t < w1) ? fabsf(r12) : 0.f;
        mx = warp_max_f(mx);                      // rows 0..W1-1 live in warps 0..W1/32-1
        if (lane == 0 && warp < (W1 + 31) / 32) sm.red[0][0][warp] = mx;
        __syncthreads();
        if (t == 0) {
            float m2 = 0.f;
#pragma unroll
            for (int q = 0; q < (W1 + 31) / 32; ++q) m2 = fmaxf(m2, sm.red[0][0][q]);
            const int fj = scale_exponent(a.kind, m2);
            a.f[j] = fj;
            sm.part_g[0] = pow2f(fj);
        }
        __syncthreads();
        if (t < W1)
            reinterpret_cast<TL*>(a.R12l)[(size_t)t + (size_t)j * W1] =
                t < w1 ? LowPrec<TL>::from_float(r12 * sm.part_g[0]) : zero;
    }
    if (!grid_barrier(a.bar, gridDim.x, a.err)) return;

    // ---- D: A2 -= (Q1l R12l) * 2^-f_j ------------------------------------------------------
    for (int i = t; i < W1 * W1; i += kNT)
        reinterpret_cast<unsigned short*>(&sm.Rl[0][0])[i] = __ldcg(reinterpret_cast<const unsigned short*>(a.R12l) + i);
    if (t < W1) sm.sc[t] = t < w2 ? pow2f(-__ldcg(a.f + t)) : 0.f;
    __syncthreads();
    {
        constexpr int kMT = kNT / 16, kNTl = W1 / 16;
        for (int tile = warp; tile < kMT * kNTl; tile += kNW) {
            const int mt = tile / kNTl, nt = tile % kNTl;
            wmma::fragment<wmma::accumulator, 16, 16, 16, float> acc;
            wmma::fill_fragment(acc, 0.f);
#pragma unroll
            for (int k0 = 0; k0 < W1; k0 += 16) {
                wmma::fragment<wmma::matrix_a, 16, 16, 16, WT, wmma::row_major> fa;
                wmma::fragment<wmma::matrix_b, 16, 16, 16, WT, wmma::col_major> fb;
                wmma::load_matrix_sync(fa, reinterpret_cast<const WT*>(&sm.QsT[mt * 16][k0]), W1 + 8);
                wmma::load_matrix_sync(fb, reinterpret_cast<const WT*>(&sm.Rl[nt * 16][k0]), W1);
                wmma::mma_sync(acc, fa, fb, acc);
            }
            wmma::store_matrix_sync(&sm.Us[mt * 16][nt * 16], acc, W1 + 4, wmma::mem_row_major);
        }
    }
    __syncthreads();
    if (valid) {
#pragma unroll
        for (int j = 0; j < W1; ++j)
            if (j < w2 && LLS_INB(row < a.ldw))
                a.W[(size_t)row + (size_t)(cA + j) * a.ldw] = fmaf(-sm.Us[t][j], sm.sc[j], av[j]);
    }
}

template <typename TL, int W1>
constexpr size_t node_smem_bytes() { return sizeof(NodeSmem<TL, W1>); }

template <typename TL, int W1>
static int node_capacity(int& cap) {
    constexpr int kMaxDev = 64;
    static int c[kMaxDev];
    static bool done[kMaxDev];
    int dev = 0;
    LLS_CUDA_TRY(cudaGetDevice(&dev));
    if (dev < 0 || dev >= kMaxDev) return LLS_ERR_UNSUPPORTED;
    if (!done[dev]) {
        const size_t smem = node_smem_bytes<TL, W1>();
        LLS_CUDA_TRY(cudaFuncSetAttribute(node_fused_kernel<TL, W1>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                          (int)smem));
        int sms = 0, per = 0;
        LLS_CUDA_TRY(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
        LLS_CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, node_fused_kernel<TL, W1>, kNT, smem));
        c[dev] = sms * per;
        done[dev] = true;
    }
    cap = c[dev];
    return LLS_OK;
}

template <typename TL, int W1>
static int launch_node(NodeArgs& a, cudaStream_t st) {
    int cap = 0;
    LLS_TRY((node_capacity<TL, W1>(cap)));
    const int P = ceil_div(a.m, kNT);
    if (P > cap) return LLS_ERR_UNSUPPORTED;
    void* args[] = {&a};
    LLS_CUDA_TRY(cudaLaunchCooperativeKernel((void*)node_fused_kernel<TL, W1>, dim3(P), dim3(kNT), args,
                                             node_smem_bytes<TL, W1>(), st));
    LLS_LAUNCH_CHECK("node_fused", st);
    return LLS_OK;
}

}  // namespace

size_t node_fused_part_floats(int m) { return (size_t)ceil_div(m, kNT) * kNodeMaxW1 * kNodeMaxW1; }

int node_fused(const NodeCall& c, cudaStream_t st) {
    if ((c.lowp != 0 && c.lowp != 1) || c.w1 > kNodeMaxW1 || c.w2 > c.w1 || c.w2 < 1) return LLS_ERR_UNSUPPORTED;
    if (node_fused_part_floats(c.m) > c.part_floats) return LLS_ERR_UNSUPPORTED;
    NodeArgs a;
    a.W = c.W; a.ldw = c.ldw; a.Wh = c.Wh; a.ldh = c.ldh;
    a.m = c.m; a.c0 = c.c0; a.w1 = c.w1; a.w2 = c.w2; a.kind = c.lowp == 0 ? 1 : 0;
    a.R = c.R; a.ldr = c.ldr; a.part = c.part; a.R12l = c.R12l; a.f = c.f;
    a.bar = c.bar; a.err = c.err;
    if (c.lowp == 0) return c.w1 <= 16 ? launch_node<__half, 16>(a, st) : launch_node<__half, 32>(a, st);
    return c.w1 <= 16 ? launch_node<__nv_bfloat16, 16>(a, st) : launch_node<__nv_bfloat16, 32>(a, st);
}

}  // namespace lls
