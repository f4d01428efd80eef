// Tensor-core products of the recursion (the projection and update of Alg. 2) on sm_103a: tcgen05.mma with the
// accumulator in tensor memory (TMEM), operands staged in shared memory by TMA.
//
//   projection  P = Q1l^T A2l       M = w1, N = w2, K = m   (both operands K-major)
//               split over K; partial tiles go to a scratch buffer and are reduced in a
//               fixed order (proj_reduce in gemm_simt.cu), which also unscales by 2^-e_j.
//   update      A2 -= (Q1l R12l) 2^-f_j   M = m, N = w2, K = w1   (Q1l is M-major)
//               the epilogue reads the FP32 A2 tile, subtracts, writes it back.
//
// Inputs are FP16 or BF16 with FP32 accumulation (kind::f16). One CTA computes one
// 128 x BN output tile (one K range): warp 0 lane 0 issues TMA loads into a STAGES-deep
// ring of shared-memory buffers, warp 1 lane 0 issues the MMAs (M = 128, N = BN, K = 16
// per instruction) and commits each stage back to the producer; after the last MMA all
// four warps read their 32 TMEM lanes (rows) and run the epilogue.
//
// Shared-memory operand layout is the canonical 128-byte-swizzled one that TMA writes:
//   K-major tile (rows x 64 elements of 2 bytes): row r at r*128 B, 8-row groups 1024 B apart
//     -> descriptor SBO = 1024 B, LBO unused (1); the k-th 16-element slice starts at +32k B.
//   M-major tile (64 K-rows x 128 M-elements): two TMA boxes of 64 M-elements, each K-row
//     128 B, box 1 at +8 KB -> descriptor LBO = 8192 B (next 64 M-elements), SBO = 1024 B
//     (next 8 K-rows); the k-th 16-row slice starts at +2048k B.
// Every wait is bounded (globaltimer); on expiry the error word is set and the CTA unwinds.
#include <cuda.h>

#include "common.cuh"
#include "kernels.cuh"
#include "tcgen05.cuh"

namespace lls {

int proj_reduce(const float* part, int splits, int w1, int w2, const int* e, const int* sq, float* R12, int ldr,
                void* R12l, int ldrl, int* f, int lowp, cudaStream_t st, const int* err);

constexpr int kTcThreads = 128;
constexpr int kTcBM = 128;
constexpr int kTcBK = 64;
constexpr int kTcStages = 4;
// Pipeline depth: 128-wide tiles keep 3 stages (97 KB of shared memory), so two CTAs share an
// SM and one CTA's epilogue (the update's read-modify-write, the projection's partial store)
// overlaps the other's main loop.
constexpr int tc_stages(int bn, int epi) { return bn == 128 ? 3 : kTcStages; }
constexpr int kTcABytes = kTcBM * kTcBK * 2;     // 16 KB
enum TcEpi { TC_EPI_PARTIAL = 0, TC_EPI_UPDATE = 1 };

struct TcArgs {
    int M, N, K;
    int k_tiles_per_split;
    uint32_t idesc;
    float* out;          // partial base (PARTIAL) or A2 (UPDATE)
    int ldo;
    const int* fexp;     // UPDATE: column exponents of R12l
    int* err;
};

template <int BN, bool A_MN, int EPI, bool F8>
__global__ void __launch_bounds__(kTcThreads, 1)
tc_gemm_kernel(const __grid_constant__ CUtensorMap tmA, const __grid_constant__ CUtensorMap tmB, TcArgs a) {
    static_assert(!(F8 && A_MN), "8-bit operands are used K-major only");
    constexpr int kKe = F8 ? 2 * kTcBK : kTcBK;   // K elements per 128-byte k-tile row
    constexpr int kStages = tc_stages(BN, EPI);
    constexpr int kBBytes = BN * kTcBK * 2;
    constexpr int kStageBytes = kTcABytes + kBBytes;
    extern __shared__ __align__(1024) uint8_t tc_smem_raw[];
    uint8_t* smem = (uint8_t*)(((uintptr_t)tc_smem_raw + 1023) & ~(uintptr_t)1023);
    uint64_t* bars = (uint64_t*)(smem + kStages * kStageBytes);
    uint32_t* tmem_slot = (uint32_t*)(bars + 2 * kStages + 1);
    const uint32_t full0 = smem_u32(bars), empty0 = smem_u32(bars + kStages);
    const uint32_t accb = smem_u32(bars + 2 * kStages);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;

    // The update walks N fastest: the CTAs that share one 128-row tile of Q1 (the larger
    // operand) run together and read it once from DRAM, then from L2.
    const int m0 = (EPI == TC_EPI_UPDATE ? blockIdx.y : blockIdx.x) * kTcBM;
    const int n0 = (EPI == TC_EPI_UPDATE ? blockIdx.x : blockIdx.y) * BN;
    const int kt_total = (a.K + kKe - 1) / kKe;
    const int kt0 = blockIdx.z * a.k_tiles_per_split;
    const int kt1 = min(kt_total, kt0 + a.k_tiles_per_split);
    const int nk = kt1 - kt0;

    if (threadIdx.x == 0) {
        for (int s = 0; s < kStages; ++s) {
            mbar_init(full0 + 8 * s, 1);
            mbar_init(empty0 + 8 * s, 1);
        }
        mbar_init(accb, 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 0) tmem_alloc(smem_u32(tmem_slot), BN);
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = *tmem_slot;
    bool ok = true;

    if (EPI == TC_EPI_UPDATE && nk > 0) {
        // Pull this CTA's FP32 tile of A2 into L2 while the main loop runs, so that the
        // epilogue's read-modify-write finds it there: one 128-byte line per 32 rows of a column.
        for (int l = threadIdx.x; l < 4 * BN; l += kTcThreads) {
            const int j = n0 + (l >> 2), i = m0 + (l & 3) * 32;
            if (j < a.N && i < a.M)
                asm volatile("prefetch.global.L2 [%0];" ::"l"(a.out + (size_t)i + (size_t)j * a.ldo));
        }
    }

    if (nk > 0) {
        if (warp == 0 && lane == 0) {
            // ---- TMA producer ----
            for (int i = 0; i < nk && ok; ++i) {
                const int s = i % kStages;
                const uint32_t ph = (i / kStages) & 1;
                if (!mbar_wait(empty0 + 8 * s, ph ^ 1, a.err)) { ok = false; break; }
                const uint32_t sa = smem_u32(smem + s * kStageBytes);
                const uint32_t sb = sa + kTcABytes;
                mbar_expect_tx(full0 + 8 * s, kStageBytes);
                const int k0 = (kt0 + i) * kKe;
                if (A_MN) {
                    tma_load_2d(sa, &tmA, m0, k0, full0 + 8 * s);
                    tma_load_2d(sa + kTcABytes / 2, &tmA, m0 + 64, k0, full0 + 8 * s);
                } else {
                    tma_load_2d(sa, &tmA, k0, m0, full0 + 8 * s);
                }
                tma_load_2d(sb, &tmB, k0, n0, full0 + 8 * s);
            }
        } else if (warp == 1 && lane == 0) {
            // ---- MMA issuer ----
            for (int i = 0; i < nk && ok; ++i) {
                const int s = i % kStages;
                const uint32_t ph = (i / kStages) & 1;
                if (!mbar_wait(full0 + 8 * s, ph, a.err)) { ok = false; break; }
                tc_fence_after();
                const uint32_t sa = smem_u32(smem + s * kStageBytes);
                const uint32_t sb = sa + kTcABytes;
#pragma unroll
                for (int kk = 0; kk < kTcBK / 16; ++kk) {
                    const uint64_t ad = A_MN ? smem_desc(sa + kk * 2048, 8192, 1024)
                                             : smem_desc(sa + kk * 32, 16, 1024);
                    const uint64_t bd = smem_desc(sb + kk * 32, 16, 1024);
                    if constexpr (F8) mma_f8(tmem, ad, bd, a.idesc, (i > 0 || kk > 0) ? 1u : 0u);
                    else mma_f16(tmem, ad, bd, a.idesc, (i > 0 || kk > 0) ? 1u : 0u);
                }
                mma_commit(empty0 + 8 * s);
            }
            if (ok) mma_commit(accb);
        }
        // ---- epilogue: all four warps, thread (warp, lane) owns tile row 32*warp + lane ----
        __syncwarp();
        const bool ready = mbar_wait(accb, 0, a.err);
        __syncwarp();
        tc_fence_after();
        if (ready && EPI == TC_EPI_PARTIAL) {
            const int i = m0 + warp * 32 + lane;
#pragma unroll 1
            for (int c = 0; c < BN / 16; ++c) {
                float v[16];
                tmem_ld16(tmem + ((uint32_t)(warp * 32) << 16) + (uint32_t)(c * 16), v);
                if (i < a.M) {
#pragma unroll
                    for (int r = 0; r < 16; ++r) {
                        const int j = n0 + c * 16 + r;
                        if (j < a.N) a.out[(size_t)blockIdx.z * a.M * a.N + (size_t)i + (size_t)j * a.M] = v[r];
                    }
                }
            }
        } else if (ready) {
            // A2 -= acc * 2^-f, 16 columns at a time. The 16 old values (and scales) of the
            // next chunk are loaded before the current chunk is stored, so each chunk costs
            // one overlapped round trip instead of one per element.
            const int i = m0 + warp * 32 + lane;
            const bool row_ok = i < a.M;
            float* orow = a.out + (size_t)(row_ok ? i : 0);
            float nxt[16], nsc[16];
#pragma unroll
            for (int r = 0; r < 16; ++r) {
                const int j = n0 + r;
                const bool in = row_ok && j < a.N;
                nxt[r] = in ? orow[(size_t)j * a.ldo] : 0.f;
                nsc[r] = in ? pow2f(-__ldg(a.fexp + j)) : 0.f;
            }
#pragma unroll 1
            for (int c = 0; c < BN / 16; ++c) {
                float cur[16], sc[16], v[16];
#pragma unroll
                for (int r = 0; r < 16; ++r) { cur[r] = nxt[r]; sc[r] = nsc[r]; }
                if (c + 1 < BN / 16) {
#pragma unroll
                    for (int r = 0; r < 16; ++r) {
                        const int j = n0 + (c + 1) * 16 + r;
                        const bool in = row_ok && j < a.N;
                        nxt[r] = in ? orow[(size_t)j * a.ldo] : 0.f;
                        nsc[r] = in ? pow2f(-__ldg(a.fexp + j)) : 0.f;
                    }
                }
                tmem_ld16(tmem + ((uint32_t)(warp * 32) << 16) + (uint32_t)(c * 16), v);
#pragma unroll
                for (int r = 0; r < 16; ++r) {
                    const int j = n0 + c * 16 + r;
                    if (row_ok && j < a.N) orow[(size_t)j * a.ldo] = fmaf(-v[r], sc[r], cur[r]);
                }
            }
        } else {
            // The pipeline gave up: let in-flight TMA writes into this CTA's shared memory
            // land before the CTA exits (bounded).
            if (warp == 0 && lane == 0) {
                const unsigned long long t0 = globaltimer_ns();
                for (int s = 0; s < kStages; ++s)
                    while (!mbar_try_wait(full0 + 8 * s, 0) && !mbar_try_wait(full0 + 8 * s, 1) &&
                           globaltimer_ns() - t0 < kSpinLimitNs) {
                    }
            }
            if (EPI == TC_EPI_UPDATE) {
                // the tile's update is unknown: write it as NaN, so the failure shows in A2
                const int i = m0 + warp * 32 + lane;
                if (i < a.M)
                    for (int j = n0; j < n0 + BN && j < a.N; ++j)
                        a.out[(size_t)i + (size_t)j * a.ldo] = __int_as_float(0x7fc00000);
            }
        }
    }
    tc_fence_before();
    __syncthreads();
    if (warp == 0) {
        tc_fence_after();
        tmem_dealloc(tmem, BN);
    }
}

// ---------------------------------------------------------------------------------------
// Host side
// ---------------------------------------------------------------------------------------
typedef CUresult (*EncodeTiledFn)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*, const cuuint64_t*,
                                  const cuuint64_t*, const cuuint32_t*, const cuuint32_t*, CUtensorMapInterleave,
                                  CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

static EncodeTiledFn encode_fn() {
    static EncodeTiledFn fn = nullptr;
    if (!fn) {
        void* p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) == cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = (EncodeTiledFn)p;
    }
    return fn;
}

int tc_make_tmap(CUtensorMap* tm, const void* base, CUtensorMapDataType dt, uint64_t esz, uint64_t inner,
                 uint64_t outer, uint64_t ld, uint32_t box_inner, uint32_t box_outer, CUtensorMapSwizzle swz) {
    EncodeTiledFn fn = encode_fn();
    if (!fn) return LLS_ERR_CUDA;
    if (((uintptr_t)base & 15) != 0 || ((ld * esz) & 15) != 0) return LLS_ERR_UNSUPPORTED;
    cuuint64_t dims[2] = {inner, outer};
    cuuint64_t strides[1] = {ld * esz};
    cuuint32_t box[2] = {box_inner, box_outer};
    cuuint32_t estr[2] = {1, 1};
    CUresult r = fn(tm, dt, 2, const_cast<void*>(base), dims, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE, swz,
                    CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    return r == CUDA_SUCCESS ? LLS_OK : LLS_ERR_CUDA;
}

// 2-D tensor map over a column-major low-precision matrix with the 128-byte swizzle.
static int make_tmap(CUtensorMap* tm, const void* base, int lowp, uint64_t inner, uint64_t outer, uint64_t ld,
                     uint32_t box_inner, uint32_t box_outer) {
    const CUtensorMapDataType dt = lowp == 0 ? CU_TENSOR_MAP_DATA_TYPE_FLOAT16
                                   : (lowp == 1 ? CU_TENSOR_MAP_DATA_TYPE_BFLOAT16 : CU_TENSOR_MAP_DATA_TYPE_UINT8);
    return tc_make_tmap(tm, base, dt, lowp == 2 ? 1 : 2, inner, outer, ld, box_inner, box_outer,
                        CU_TENSOR_MAP_SWIZZLE_128B);
}

uint32_t tc_make_idesc(int lowp, int bn, bool a_mn) {
    const uint32_t fmt = lowp == 1 ? 1u : 0u;       // kind::f16: 0 = F16, 1 = BF16; kind::f8f6f4: 0 = E4M3
    uint32_t d = 0;
    d |= 1u << 4;                                    // D = F32
    d |= fmt << 7;                                   // A type
    d |= fmt << 10;                                  // B type
    d |= (a_mn ? 1u : 0u) << 15;                     // A major (0 = K, 1 = MN)
    d |= (uint32_t)(bn >> 3) << 17;                  // N / 8
    d |= (uint32_t)(kTcBM >> 4) << 24;               // M / 16
    return d;
}

static uint32_t make_idesc(int lowp, int bn, bool a_mn) { return tc_make_idesc(lowp, bn, a_mn); }

static int pick_bn(int n) { return n <= 64 ? 64 : 128; }

template <int BN, bool A_MN, int EPI, bool F8>
static int launch_tc(const CUtensorMap& tA, const CUtensorMap& tB, const TcArgs& a, dim3 grid, cudaStream_t st) {
    constexpr int smem = tc_stages(BN, EPI) * (kTcABytes + BN * kTcBK * 2) + 1024 + 256;
    auto k = tc_gemm_kernel<BN, A_MN, EPI, F8>;
    static bool attr = false;
    if (!attr) {
        LLS_CUDA_TRY(cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, smem));
        attr = true;
    }
    k<<<grid, kTcThreads, smem, st>>>(tA, tB, a);
    LLS_LAUNCH_CHECK(EPI == TC_EPI_PARTIAL ? "tc_projection" : "tc_update", st);
    return LLS_OK;
}

template <bool A_MN, int EPI, bool F8 = false>
static int launch_bn(int bn, const CUtensorMap& tA, const CUtensorMap& tB, const TcArgs& a, dim3 grid, cudaStream_t st) {
    if (bn == 64) return launch_tc<64, A_MN, EPI, F8>(tA, tB, a, grid, st);
    if (bn == 128) return launch_tc<128, A_MN, EPI, F8>(tA, tB, a, grid, st);
    return launch_tc<256, A_MN, EPI, F8>(tA, tB, a, grid, st);
}

static int sm_count() {
    static int sms = 0;
    if (!sms) {
        int dev = 0;
        if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
            sms = 148;
    }
    return sms;
}

static void proj_split(int m, int w1, int w2, int& splits, int& ktps, int lowp = 0) {
    const int bn = pick_bn(w2);
    const int tiles = ceil_div(w1, kTcBM) * ceil_div(w2, bn);
    const int kt = ceil_div(m, lowp == 2 ? 2 * kTcBK : kTcBK);
    int want = ceil_div(2 * sm_count(), tiles);             // about two waves of CTAs
    int maxs = kt / 8 > 0 ? kt / 8 : 1;                      // at least 8 K tiles per CTA
    splits = want < maxs ? want : maxs;
    if (splits < 1) splits = 1;
    ktps = ceil_div(kt, splits);
    splits = ceil_div(kt, ktps);
}

void proj_split_persistent(int m, int w1, int w2, int& splits, int& ktps);
bool projection_persistent_applies(int lowp, int w1, int w2);
int gemm_projection_persistent(const ProjCall& c, cudaStream_t st);
int gemm_update_persistent(const UpdCall& c, cudaStream_t st);

// Partial sums of the projection: room for either kernel's K split.
size_t proj_partial_floats(int m, int w1, int w2) {
    int splits, ktps, ps, pk;
    proj_split(m, w1, w2, splits, ktps);
    proj_split_persistent(m, w1, w2, ps, pk);
    return (size_t)(splits > ps ? splits : ps) * w1 * w2;
}

int gemm_projection(const ProjCall& c, cudaStream_t st) {
    if (c.gemm_kernel == 0 && projection_persistent_applies(c.lowp, c.w1, c.w2)) {
        const int r = gemm_projection_persistent(c, st);
        if (r != LLS_ERR_UNSUPPORTED) return r;
    }
    int splits, ktps;
    proj_split(c.m, c.w1, c.w2, splits, ktps, c.lowp);
    if ((size_t)splits * c.w1 * c.w2 > c.part_floats) return LLS_ERR_WORKSPACE;
    const int bn = pick_bn(c.w2);
    const uint32_t bk = c.lowp == 2 ? 2 * kTcBK : kTcBK;     // 128-byte rows
    CUtensorMap tA, tB;
    LLS_TRY(make_tmap(&tA, c.Q1l, c.lowp, (uint64_t)c.m, (uint64_t)c.w1, (uint64_t)c.ldh, bk, kTcBM));
    LLS_TRY(make_tmap(&tB, c.A2l, c.lowp, (uint64_t)c.m, (uint64_t)c.w2, (uint64_t)c.ldh, bk, (uint32_t)bn));
    TcArgs a;
    a.M = c.w1; a.N = c.w2; a.K = c.m; a.k_tiles_per_split = ktps;
    a.idesc = make_idesc(c.lowp, bn, false);
    a.out = c.part; a.ldo = c.w1; a.fexp = nullptr; a.err = c.err;
    dim3 grid(ceil_div(c.w1, kTcBM), ceil_div(c.w2, bn), splits);
    if (c.lowp == 2) LLS_TRY((launch_bn<false, TC_EPI_PARTIAL, true>(bn, tA, tB, a, grid, st)));
    else LLS_TRY((launch_bn<false, TC_EPI_PARTIAL>(bn, tA, tB, a, grid, st)));
    return proj_reduce(c.part, splits, c.w1, c.w2, c.e, c.sq, c.R12, c.ldr, c.R12l, c.ldrl, c.f, c.lowp, st, c.err);
}

int gemm_update(const UpdCall& c, cudaStream_t st) {
    {
        const int r = gemm_update_persistent(c, st);
        if (r != LLS_ERR_UNSUPPORTED) return r;
    }
    const int bn = c.w2 <= 64 ? 64 : 128;
    if (c.lowp == 2) {
        // FP8: A = Q1 row-major (K-major, rows of ldq bytes), B = R12l (K-major)
        if (!c.QT) return LLS_ERR_UNSUPPORTED;
        CUtensorMap tA, tB;
        LLS_TRY(make_tmap(&tA, c.QT, 2, (uint64_t)c.w1, (uint64_t)c.m, (uint64_t)c.ldq, 2 * kTcBK, kTcBM));
        LLS_TRY(make_tmap(&tB, c.R12l, 2, (uint64_t)c.w1, (uint64_t)c.w2, (uint64_t)c.ldrl, 2 * kTcBK, (uint32_t)bn));
        TcArgs a;
        a.M = c.m; a.N = c.w2; a.K = c.w1; a.k_tiles_per_split = ceil_div(c.w1, 2 * kTcBK);
        a.idesc = make_idesc(2, bn, false);
        a.out = c.A2; a.ldo = c.ldw; a.fexp = c.f; a.err = c.err;
        dim3 grid(ceil_div(c.w2, bn), ceil_div(c.m, kTcBM), 1);
        return launch_bn<false, TC_EPI_UPDATE, true>(bn, tA, tB, a, grid, st);
    }
    CUtensorMap tA, tB;
    LLS_TRY(make_tmap(&tA, c.Q1l, c.lowp, (uint64_t)c.m, (uint64_t)c.w1, (uint64_t)c.ldh, 64, kTcBK));
    LLS_TRY(make_tmap(&tB, c.R12l, c.lowp, (uint64_t)c.w1, (uint64_t)c.w2, (uint64_t)c.ldrl, kTcBK, (uint32_t)bn));
    TcArgs a;
    a.M = c.m; a.N = c.w2; a.K = c.w1; a.k_tiles_per_split = ceil_div(c.w1, kTcBK);
    a.idesc = make_idesc(c.lowp, bn, true);
    a.out = c.A2; a.ldo = c.ldw; a.fexp = c.f; a.err = c.err;
    dim3 grid(ceil_div(c.w2, bn), ceil_div(c.m, kTcBM), 1);
    return launch_bn<true, TC_EPI_UPDATE>(bn, tA, tB, a, grid, st);
}

}  // namespace lls
