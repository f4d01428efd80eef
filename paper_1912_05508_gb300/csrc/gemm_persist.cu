// Persistent tensor-core products for the wide recursion nodes of Alg. 2 (FP16 / BF16 operands,
// FP32 accumulation in tensor memory), one CTA per SM looping over output tiles:
//
//   update      A2 -= (Q1l R12l) 2^-f_j      M = m, N = w2, K = w1 (Q1l M-major, R12l K-major)
//   projection  part[s] = Q1l^T A2l           M = w1, N = w2, K-split s of K = m (both K-major)
//
// Warp roles (256 threads):
//   warp 0      TMA loads of the operand tiles into a ring of shared-memory stages;
//   warp 1      tcgen05.mma issue (one thread) into one of TWO accumulators in TMEM (2 x 128
//               columns), so the epilogue of tile t overlaps the MMAs of tile t + 1;
//   warp 2      (update) TMA loads of the FP32 A2 tile, 32 columns at a time, into a ring of
//               chunk buffers, ahead of the epilogue;
//   warps 4-7   epilogue, one TMEM lane (tile row) per thread: the update subtracts the product
//               from the A2 chunk in shared memory and one thread writes the chunk back with a
//               TMA store; the projection stores its partial tile directly.
// Every mbarrier wait is bounded (about 2 s of %globaltimer): on expiry the error word is set and
// the roles fall through to the end; the epilogue then overwrites the CTA's update tiles with NaN
// (projection partials are turned into NaN by the reduction that reads the error word), the
// issuing threads wait (bounded) for their copies and MMAs still in flight, and TMEM is freed.
#include "common.cuh"
#include "kernels.cuh"
#include "tcgen05.cuh"

namespace lls {

int proj_reduce(const float* part, int splits, int w1, int w2, const int* e, const int* sq, float* R12, int ldr,
                void* R12l, int ldrl, int* f, int lowp, cudaStream_t st, const int* err);

namespace {

constexpr int kPM = 128;                     // tile rows (M)
constexpr int kPK = 64;                      // K per stage: 128-byte rows of 2-byte elements
constexpr int kPThreads = 256;
constexpr int kABytes = kPM * kPK * 2;       // 16 KB

enum { PE_PARTIAL = 0, PE_UPDATE = 1 };

// Tile width BN (128 or 256 columns: one accumulator of BN TMEM columns, two of them), pipeline
// depth and A2 chunk buffers, sized to the 227 KB of shared memory a CTA may hold. Wider tiles
// halve the operand traffic from L2 per flop, which the 128 x 128 tiles are bound by.
// The wide update keeps four operand stages (three left the tensor pipe idle half the time
// while operands arrived) and moves A2 in 16-column chunks through four buffers.
template <int EPI, int BN> struct PCfg {
    static constexpr int bbytes = BN * kPK * 2;
    static constexpr int stage_bytes = kABytes + bbytes;
    static constexpr int stages = EPI == PE_UPDATE ? 4 : (BN == 256 ? 4 : 6);
    static constexpr int ccols = (EPI == PE_UPDATE && BN == 256) ? 16 : 32;   // A2 columns per chunk
    static constexpr int cbytes = kPM * ccols * 4;
    static constexpr int ring = EPI == PE_UPDATE ? (BN == 256 ? 4 : 6) : 0;
    static constexpr int chunks = BN / ccols;
};

template <int EPI, int BN>
constexpr int p_smem_bytes() {
    using C = PCfg<EPI, BN>;
    return 1024 + C::stages * C::stage_bytes + C::ring * C::cbytes + 512;   // + barriers
}

struct PArgs {
    int M, N;
    int tiles_m, tiles_n, splits;
    int ktotal, ktiles;        // K tiles in all, and per split
    uint32_t idesc;
    float* out;                // PARTIAL: partial sums [split][N][M]; UPDATE: A2 (poisoned on failure)
    int ldo;
    const int* fexp;           // UPDATE: column exponents of R12l
    int* err;
};

template <int BN>
__device__ __forceinline__ void decode_unit(const PArgs& a, int u, int& m0, int& n0, int& kt0, int& kt1, int& s) {
    const int tiles = a.tiles_m * a.tiles_n;
    s = u / tiles;
    const int t = u - s * tiles;
    m0 = (t / a.tiles_n) * kPM;     // N fastest: the tiles that share a block of rows of the A
    n0 = (t % a.tiles_n) * BN;      // operand run at the same time and read it from L2
    kt0 = s * a.ktiles;
    kt1 = min(a.ktotal, kt0 + a.ktiles);
}

// Bounded wait for the copies a thread issued into `count` ring slots: slot i received the
// issue of sequence number last(i), so its phase ((last / count) & 1) must have completed.
__device__ __forceinline__ void drain_ring(uint32_t full0, int count, uint32_t issued) {
    const unsigned long long t0 = globaltimer_ns();
    for (int i = 0; i < count && (uint32_t)i < issued; ++i) {
        const uint32_t last = issued - 1 - ((issued - 1 - i) % count);
        const uint32_t ph = (last / count) & 1;
        while (!mbar_try_wait(full0 + 8 * i, ph) && globaltimer_ns() - t0 < kSpinLimitNs) {
        }
    }
}

template <int EPI, bool A_MN, int BN>
__global__ void __launch_bounds__(kPThreads, 1)
tc_persist_kernel(const __grid_constant__ CUtensorMap tmA, const __grid_constant__ CUtensorMap tmB,
                  const __grid_constant__ CUtensorMap tmC, PArgs a) {
    using Cfg = PCfg<EPI, BN>;
    constexpr int S = Cfg::stages;
    constexpr int NR = Cfg::ring > 0 ? Cfg::ring : 1;
    constexpr int kStageBytes = Cfg::stage_bytes;
    constexpr int kCChunks = Cfg::chunks;
    constexpr int kCCols = Cfg::ccols;
    constexpr int kCBytes = Cfg::cbytes;
    constexpr int kPN = BN;
    extern __shared__ __align__(1024) uint8_t p_smem_raw[];
    uint8_t* smem = (uint8_t*)(((uintptr_t)p_smem_raw + 1023) & ~(uintptr_t)1023);
    uint8_t* cring = smem + S * kStageBytes;
    uint64_t* bars = (uint64_t*)(cring + Cfg::ring * Cfg::cbytes);
    // full[S], empty[S], tfull[2], tempty[2], cfull[NR], cempty[NR], cdone[NR], mmadone, sdone
    const uint32_t full0 = smem_u32(bars), empty0 = full0 + 8 * S;
    const uint32_t tfull0 = empty0 + 8 * S, tempty0 = tfull0 + 16;
    const uint32_t cfull0 = tempty0 + 16, cempty0 = cfull0 + 8 * NR, cdone0 = cempty0 + 8 * NR;
    const uint32_t mmadone = cdone0 + 8 * NR, sdone = mmadone + 8;
    uint32_t* tmem_slot = (uint32_t*)(bars + 2 * S + 4 + 3 * NR + 2);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int units = a.tiles_m * a.tiles_n * a.splits;

    if (threadIdx.x == 0) {
        for (int i = 0; i < S; ++i) {
            mbar_init(full0 + 8 * i, 1);
            mbar_init(empty0 + 8 * i, 1);
        }
        for (int i = 0; i < 2; ++i) {
            mbar_init(tfull0 + 8 * i, 1);
            mbar_init(tempty0 + 8 * i, 4);      // one arrival per epilogue warp
        }
        for (int i = 0; i < NR; ++i) {
            mbar_init(cfull0 + 8 * i, 1);
            mbar_init(cempty0 + 8 * i, 1);
            mbar_init(cdone0 + 8 * i, 4);       // every epilogue warp wrote its rows of the chunk
        }
        mbar_init(mmadone, 1);
        mbar_init(sdone, 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 1) tmem_alloc(smem_u32(tmem_slot), 2 * kPN);
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = *tmem_slot;

    if (warp == 0 && lane == 0) {
        // ---- operand producer ----
        uint32_t it = 0;
        bool ok = true;
        for (int u = blockIdx.x; u < units && ok; u += gridDim.x) {
            int m0, n0, kt0, kt1, s;
            decode_unit<BN>(a, u, m0, n0, kt0, kt1, s);
            for (int kt = kt0; kt < kt1; ++kt, ++it) {
                const int st = it % S;
                const uint32_t ph = (it / S) & 1;
                if (!mbar_wait(empty0 + 8 * st, ph ^ 1, a.err)) { ok = false; break; }
                const uint32_t sa = smem_u32(smem + st * kStageBytes), sb = sa + kABytes;
                mbar_expect_tx(full0 + 8 * st, kStageBytes);
                const int k0 = kt * kPK;
                if (A_MN) {
                    tma_load_2d(sa, &tmA, m0, k0, full0 + 8 * st);
                    tma_load_2d(sa + kABytes / 2, &tmA, m0 + 64, k0, full0 + 8 * st);
                } else {
                    tma_load_2d(sa, &tmA, k0, m0, full0 + 8 * st);
                }
                tma_load_2d(sb, &tmB, k0, n0, full0 + 8 * st);
            }
        }
        drain_ring(full0, S, it);       // no copy into shared memory may outlive the CTA
    } else if (warp == 1) {
        if (lane == 0) {
            // ---- MMA issuer ----
            uint32_t it = 0;
            bool ok = true;
            int lt = 0;
            for (int u = blockIdx.x; u < units && ok; u += gridDim.x, ++lt) {
                int m0, n0, kt0, kt1, s;
                decode_unit<BN>(a, u, m0, n0, kt0, kt1, s);
                const int acc = lt & 1;
                const uint32_t use = (uint32_t)(lt >> 1);
                if (!mbar_wait(tempty0 + 8 * acc, (use & 1) ^ 1, a.err)) { ok = false; break; }
                tc_fence_after();
                const uint32_t d = tmem + (uint32_t)(acc * kPN);
                for (int kt = kt0; kt < kt1; ++kt, ++it) {
                    const int st = it % S;
                    const uint32_t ph = (it / S) & 1;
                    if (!mbar_wait(full0 + 8 * st, ph, a.err)) { ok = false; break; }
                    tc_fence_after();
                    const uint32_t sa = smem_u32(smem + st * kStageBytes), sb = sa + kABytes;
#pragma unroll
                    for (int kk = 0; kk < kPK / 16; ++kk) {
                        const uint64_t ad = A_MN ? smem_desc(sa + kk * 2048, 8192, 1024) : smem_desc(sa + kk * 32, 16, 1024);
                        const uint64_t bd = smem_desc(sb + kk * 32, 16, 1024);
                        mma_f16(d, ad, bd, a.idesc, (kt > kt0 || kk > 0) ? 1u : 0u);
                    }
                    mma_commit(empty0 + 8 * st);
                }
                if (!ok) break;
                mma_commit(tfull0 + 8 * acc);
            }
            // every MMA issued has completed before the accumulators are released
            mma_commit(mmadone);
            const unsigned long long t0 = globaltimer_ns();
            while (!mbar_try_wait(mmadone, 0) && globaltimer_ns() - t0 < kSpinLimitNs) {
            }
        }
        __syncwarp();
    } else if (EPI == PE_UPDATE && warp == 2 && lane == 0) {
        // ---- A2 chunk loader ----
        uint32_t cc = 0;
        bool ok = true;
        for (int u = blockIdx.x; u < units && ok; u += gridDim.x) {
            int m0, n0, kt0, kt1, s;
            decode_unit<BN>(a, u, m0, n0, kt0, kt1, s);
            for (int c = 0; c < kCChunks; ++c, ++cc) {
                const int slot = cc % NR;
                const uint32_t ph = (cc / NR) & 1;
                if (!mbar_wait(cempty0 + 8 * slot, ph ^ 1, a.err)) { ok = false; break; }
                mbar_expect_tx(cfull0 + 8 * slot, kCBytes);
                tma_load_2d(smem_u32(cring + slot * kCBytes), &tmC, m0, n0 + c * kCCols, cfull0 + 8 * slot);
            }
        }
        drain_ring(cfull0, NR, cc);
    } else if (warp >= 4) {
        // ---- epilogue: thread = tile row 32 (warp - 4) + lane = its TMEM lane ----
        const int e = warp - 4, r = 32 * e + lane;
        bool ok = true;
        int lt = 0;
        uint32_t cc = 0;
        const bool storer = (warp == 4 && lane == 0);
        for (int u = blockIdx.x; u < units; u += gridDim.x, ++lt) {
            int m0, n0, kt0, kt1, s;
            decode_unit<BN>(a, u, m0, n0, kt0, kt1, s);
            const int acc = lt & 1;
            const uint32_t use = (uint32_t)(lt >> 1);
            if (ok && !mbar_wait(tfull0 + 8 * acc, use & 1, a.err)) ok = false;
            tc_fence_after();
            const uint32_t tbase = tmem + ((uint32_t)(32 * e) << 16) + (uint32_t)(acc * kPN);
#pragma unroll 1
            for (int c = 0; c < kCChunks; ++c, ++cc) {
                float v[kCCols];
                if (ok) {
                    if constexpr (kCCols == 32) tmem_ld32(tbase + (uint32_t)(c * kCCols), v);
                    else tmem_ld16(tbase + (uint32_t)(c * kCCols), v);
                }
                if constexpr (EPI == PE_UPDATE) {
                    const int slot = cc % NR;
                    const uint32_t ph = (cc / NR) & 1;
                    if (ok && !mbar_wait(cfull0 + 8 * slot, ph, a.err)) ok = false;
                    float* cb = reinterpret_cast<float*>(cring + slot * kCBytes);   // [chunk columns][128 rows]
                    if (ok) {
#pragma unroll
                        for (int j = 0; j < kCCols; ++j) {
                            const int col = n0 + c * kCCols + j;
                            const float sc = col < a.N ? pow2f(-__ldg(a.fexp + col)) : 0.f;
                            cb[j * kPM + r] = fmaf(-v[j], sc, cb[j * kPM + r]);
                        }
                    }
                    fence_proxy_async_smem();
                    __syncwarp();
                    if (lane == 0) mbar_arrive(cdone0 + 8 * slot);
                    if (storer) {
                        // the chunk is complete once all four warps arrived; then write it back
                        if (ok && !mbar_wait(cdone0 + 8 * slot, ph, a.err)) ok = false;
                        // a TMA store must not start at a negative coordinate (one past the
                        // edge is clipped by the unit)
                        if (ok && LLS_INB(m0 >= 0 && m0 < a.M && n0 + c * kCCols >= 0)) {
                            tma_store_2d(&tmC, m0, n0 + c * kCCols, smem_u32(cb));
                            bulk_commit();
                        }
                        // the previous chunk's store has read its buffer: hand that buffer back
                        bulk_wait_read<1>();
                        if (cc > 0) mbar_arrive(cempty0 + 8 * ((cc - 1) % NR));
                    }
                } else {
                    if (ok) {
                        const int row = m0 + r;
                        float* o = a.out + (size_t)s * a.M * a.N;
                        if (row < a.M && LLS_INB(s >= 0 && s < a.splits && row >= 0)) {
#pragma unroll
                            for (int j = 0; j < kCCols; ++j) {
                                const int col = n0 + c * kCCols + j;
                                if (col < a.N) o[(size_t)row + (size_t)col * a.M] = v[j];
                            }
                        }
                    }
                }
            }
            // this accumulator's TMEM columns are free once all four warps have read them
            tc_fence_before();
            __syncwarp();
            if (lane == 0) mbar_arrive(tempty0 + 8 * acc);
        }
        if constexpr (EPI == PE_UPDATE) {
            if (storer) {
                bulk_wait_all<0>();
                if (cc > 0) mbar_arrive(cempty0 + 8 * ((cc - 1) % NR));
                mbar_arrive(sdone);          // this CTA's stores have all landed
            }
            if (*(volatile int*)a.err != DEV_OK) {
                // the update of this CTA's tiles is unknown: write them as NaN, after its stores
                const unsigned long long t0 = globaltimer_ns();
                while (!mbar_try_wait(sdone, 0) && globaltimer_ns() - t0 < kSpinLimitNs) {
                }
                for (int u = blockIdx.x; u < units; u += gridDim.x) {
                    int m0, n0, kt0, kt1, s;
                    decode_unit<BN>(a, u, m0, n0, kt0, kt1, s);
                    const int row = m0 + r;
                    if (row < a.M)
                        for (int j = n0; j < n0 + kPN && j < a.N; ++j)
                            a.out[(size_t)row + (size_t)j * a.ldo] = __int_as_float(0x7fc00000);
                }
            }
        }
    }
    tc_fence_before();
    __syncthreads();
    if (warp == 1) {
        tc_fence_after();
        tmem_dealloc(tmem, 2 * kPN);
    }
}

int sms_of_device() {
    static int sms[64];
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return 0;
    if (!sms[dev] && cudaDeviceGetAttribute(&sms[dev], cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return 0;
    return sms[dev];
}

template <int EPI, bool A_MN, int BN>
int launch_persist(const CUtensorMap& tA, const CUtensorMap& tB, const CUtensorMap& tC, const PArgs& a,
                   cudaStream_t st) {
    constexpr int smem = p_smem_bytes<EPI, BN>();
    static_assert(smem <= 232448, "shared memory of one CTA");
    auto k = tc_persist_kernel<EPI, A_MN, BN>;
    static bool attr[64];
    int dev = 0;
    LLS_CUDA_TRY(cudaGetDevice(&dev));
    if (dev < 0 || dev >= 64) return LLS_ERR_UNSUPPORTED;
    if (!attr[dev]) {
        LLS_CUDA_TRY(cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, smem));
        attr[dev] = true;
    }
    const int sms = sms_of_device();
    if (sms <= 0) return LLS_ERR_CUDA;
    const int units = a.tiles_m * a.tiles_n * a.splits;
    const int grid = units < sms ? units : sms;
    k<<<grid, kPThreads, smem, st>>>(tA, tB, tC, a);
    LLS_LAUNCH_CHECK(EPI == PE_PARTIAL ? "tc_projection_persistent" : "tc_update_persistent", st);
    return LLS_OK;
}

}  // namespace

// The update on the persistent kernel; LLS_ERR_UNSUPPORTED (nothing launched) when the shape or
// the operands' alignment does not fit it (the caller then uses the one-tile-per-CTA kernel).
template <int BN>
static int update_persistent_bn(const UpdCall& c, cudaStream_t st) {
    const CUtensorMapDataType dt = c.lowp == 0 ? CU_TENSOR_MAP_DATA_TYPE_FLOAT16 : CU_TENSOR_MAP_DATA_TYPE_BFLOAT16;
    CUtensorMap tA, tB, tC;
    if (tc_make_tmap(&tA, c.Q1l, dt, 2, (uint64_t)c.m, (uint64_t)c.w1, (uint64_t)c.ldh, 64, kPK,
                     CU_TENSOR_MAP_SWIZZLE_128B) != LLS_OK ||
        tc_make_tmap(&tB, c.R12l, dt, 2, (uint64_t)c.w1, (uint64_t)c.w2, (uint64_t)c.ldrl, kPK, BN,
                     CU_TENSOR_MAP_SWIZZLE_128B) != LLS_OK ||
        tc_make_tmap(&tC, c.A2, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 4, (uint64_t)c.m, (uint64_t)c.w2, (uint64_t)c.ldw,
                     kPM, PCfg<PE_UPDATE, BN>::ccols, CU_TENSOR_MAP_SWIZZLE_NONE) != LLS_OK)
        return LLS_ERR_UNSUPPORTED;
    PArgs a;
    a.M = c.m; a.N = c.w2;
    a.tiles_m = ceil_div(c.m, kPM); a.tiles_n = ceil_div(c.w2, BN); a.splits = 1;
    a.ktotal = ceil_div(c.w1, kPK); a.ktiles = a.ktotal;
    a.idesc = tc_make_idesc(c.lowp, BN, true);
    a.out = c.A2; a.ldo = c.ldw; a.fexp = c.f; a.err = c.err;
    return launch_persist<PE_UPDATE, true, BN>(tA, tB, tC, a, st);
}

// The update on the persistent kernel; LLS_ERR_UNSUPPORTED (nothing launched) when the shape or
// the operands' alignment does not fit it (the caller then uses the one-tile-per-CTA kernel).
// Nodes at least 256 columns wide take 128 x 256 tiles, narrower ones 128 x 128.
int gemm_update_persistent(const UpdCall& c, cudaStream_t st) {
    if (c.gemm_kernel == 1 || (c.lowp != 0 && c.lowp != 1) || c.w2 < 128 || c.w1 < kPK) return LLS_ERR_UNSUPPORTED;
    if (((uintptr_t)c.A2 & 15) != 0 || (c.ldw & 3) != 0) return LLS_ERR_UNSUPPORTED;
    return c.w2 >= 256 ? update_persistent_bn<256>(c, st) : update_persistent_bn<128>(c, st);
}

// K splits of the persistent projection: the work of the most loaded CTA (whole units per CTA
// times the K tiles of a unit) plus the partial sums' round trip through memory (written here,
// read by the fixed-order reduction), both in units of one K tile of MMAs; at most 8 splits and
// at least 8 K tiles per split. Ties go to fewer splits.
static int proj_bn(int w2) { return w2 >= 256 ? 256 : 128; }

void proj_split_persistent(int m, int w1, int w2, int& splits, int& ktps) {
    const int sms = sms_of_device() > 0 ? sms_of_device() : 148;
    const int bn = proj_bn(w2);
    const long long tiles = (long long)ceil_div(w1, kPM) * ceil_div(w2, bn);
    const int kt = ceil_div(m, kPK);
    // one K tile of a 128 x bn unit moves (128 + bn) x 64 x 2 bytes through the tensor cores in
    // about bn / 128 x 0.15 us; a split's partial tile set is w1 x w2 x 8 bytes of traffic at
    // about 5 TB/s, spread over all SMs
    const double ktile_us = 0.15 * bn / 128.0;
    const double split_units = ((double)w1 * w2 * 8.0 / 5.0e12 * 1e6) / ktile_us;
    int best_s = 1;
    double best = -1.0;
    for (int s = 1; s <= 8 && (s == 1 || kt / s >= 8); ++s) {
        const int per = ceil_div(kt, s);
        const int ss = ceil_div(kt, per);                 // splits actually non-empty
        const long long units = tiles * ss;
        const double cost = (double)((units + sms - 1) / sms) * per + split_units * ss;
        if (best < 0.0 || cost < best) { best = cost; best_s = ss; }
    }
    ktps = ceil_div(kt, best_s);
    splits = ceil_div(kt, ktps);
}

bool projection_persistent_applies(int lowp, int w1, int w2) {
    return (lowp == 0 || lowp == 1) && w1 >= kPM && w2 >= 128;
}

template <int BN>
static int projection_persistent_bn(const ProjCall& c, int splits, int ktps, cudaStream_t st) {
    const CUtensorMapDataType dt = c.lowp == 0 ? CU_TENSOR_MAP_DATA_TYPE_FLOAT16 : CU_TENSOR_MAP_DATA_TYPE_BFLOAT16;
    CUtensorMap tA, tB;
    if (tc_make_tmap(&tA, c.Q1l, dt, 2, (uint64_t)c.m, (uint64_t)c.w1, (uint64_t)c.ldh, kPK, kPM,
                     CU_TENSOR_MAP_SWIZZLE_128B) != LLS_OK ||
        tc_make_tmap(&tB, c.A2l, dt, 2, (uint64_t)c.m, (uint64_t)c.w2, (uint64_t)c.ldh, kPK, BN,
                     CU_TENSOR_MAP_SWIZZLE_128B) != LLS_OK)
        return LLS_ERR_UNSUPPORTED;
    PArgs a;
    a.M = c.w1; a.N = c.w2;
    a.tiles_m = ceil_div(c.w1, kPM); a.tiles_n = ceil_div(c.w2, BN); a.splits = splits;
    a.ktotal = ceil_div(c.m, kPK); a.ktiles = ktps;
    a.idesc = tc_make_idesc(c.lowp, BN, false);
    a.out = c.part; a.ldo = c.w1; a.fexp = nullptr; a.err = c.err;
    return launch_persist<PE_PARTIAL, false, BN>(tA, tB, tA, a, st);
}

int gemm_projection_persistent(const ProjCall& c, cudaStream_t st) {
    if (c.gemm_kernel != 0 || !projection_persistent_applies(c.lowp, c.w1, c.w2)) return LLS_ERR_UNSUPPORTED;
    int splits, ktps;
    proj_split_persistent(c.m, c.w1, c.w2, splits, ktps);
    if ((size_t)splits * c.w1 * c.w2 > c.part_floats) return LLS_ERR_WORKSPACE;
    const int r = proj_bn(c.w2) == 256 ? projection_persistent_bn<256>(c, splits, ktps, st)
                                       : projection_persistent_bn<128>(c, splits, ktps, st);
    LLS_TRY(r);
    return proj_reduce(c.part, splits, c.w1, c.w2, c.e, c.sq, c.R12, c.ldr, c.R12l, c.ldrl, c.f, c.lowp, st, c.err);
}

}  // namespace lls
