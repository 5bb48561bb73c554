// Reduced-precision all-pairs correlation on the 5th-generation tensor cores
// (project addition to the paper's Section 4.2 focus refinement: the brick
// pair's Pearson / Spearman values as one contraction Z_A Z_B^T of unit-norm
// standardized member vectors).
//
// Operands are K-major planes [rows][K] of BF16, or FP8 E4M3 scaled per point
// (value * 448 / max|value|), loaded by TMA with 128-byte swizzle into a
// 4-stage shared-memory ring. One elected thread issues tcgen05.mma
// (M = 128, N = 256, FP32 accumulation in TMEM, two accumulator buffers so the
// epilogue of one tile overlaps the MMAs of the next). Eight epilogue warps
// read TMEM with tcgen05.ld and emit, per output row and 32-column chunk, the
// max and min of the approximate correlations (FP8, and BF16 integer ranks:
// rescaled by the two per-point inverse scales). No per-pair value is stored:
// the chunk extremes select the candidates that are re-evaluated exactly
// afterwards. Optionally the epilogue also counts both sides' extremes into
// the selection's first-level histogram (top 11 bits of their order-preserving
// keys, in shared memory, added to global memory once per CTA).
//
// Warp roles (320 threads, one CTA per SM, persistent over tiles):
//   warp 0  TMA producer        warp 1  TMEM allocation + MMA issuer
//   warps 2-9  epilogue (warp w reads TMEM lanes 32*(w%4) .. +31, warps 2-5
//              the tile's first 128 columns, warps 6-9 the last 128)
// Every mbarrier wait is bounded (wall clock); on timeout the CTA records
// DEV_TIMEOUT, the other roles leave their loops, in-flight copies and MMAs
// are drained with bounded waits, and TMEM is freed before returning.
#include <cuda.h>

#include "device.cuh"
#include "internal.cuh"
#include "tc_dev.cuh"

namespace cc {
namespace tc {

constexpr int TM = 128, TN = 256, STAGES = 4;
constexpr int A_BYTES = TM * 128, B_BYTES = TN * 128, STAGE_BYTES = A_BYTES + B_BYTES;
constexpr int THREADS = 320;  // TMA warp, MMA warp, 8 epilogue warps
constexpr int EPI = 256;      // epilogue threads
constexpr int TMEM_COLS = 512;  // two 256-column fp32 accumulators
// first-level histogram of the candidate selection: the top 11 bits of the
// order-preserving key (the selection's second level resolves 12 more)
constexpr int HIST_SHIFT = 21, HIST_BINS = 1 << (32 - HIST_SHIFT);

// order-preserving unsigned key of a float (-0 and +0 map to one key)
__device__ __forceinline__ unsigned order_key(float v) {
    const unsigned b = __float_as_uint(v + 0.0f);
    return (b & 0x80000000u) ? ~b : (b | 0x80000000u);
}

// Instruction descriptor: FP32 accumulator, A/B BF16 (kind::f16) or E4M3
// (kind::f8f6f4), both K-major, N = 256, M = 128.
template <bool FP8>
__host__ __device__ constexpr uint32_t idesc() {
    return (1u << 4) | ((FP8 ? 0u : 1u) << 7) | ((FP8 ? 0u : 1u) << 10) | ((uint32_t)(TN >> 3) << 17) |
           ((uint32_t)(TM >> 4) << 24);
}
template <bool FP8>
__device__ __forceinline__ void mma(uint32_t d, uint64_t a, uint64_t b, uint32_t accum) {
    if constexpr (FP8) {
        asm volatile(
            "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
            "tcgen05.mma.cta_group::1.kind::f8f6f4 [%0], %1, %2, %3, p;\n\t}" ::"r"(d),
            "l"(a), "l"(b), "r"(idesc<FP8>()), "r"(accum));
    } else {
        asm volatile(
            "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
            "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(d),
            "l"(a), "l"(b), "r"(idesc<FP8>()), "r"(accum));
    }
}

template <bool FP8, bool SCALED>
__global__ void __launch_bounds__(THREADS, 1)
    k_tc_chunk_extremes(const __grid_constant__ CUtensorMap tma,
                        const __grid_constant__ CUtensorMap tmb, int num_kb, int64_t na,
                        int64_t nb, int tiles_m, int tiles_n, int self,
                        const float* __restrict__ inv_sa, const float* __restrict__ inv_sb,
                        float* __restrict__ cmax, float* __restrict__ cmin, int64_t na_pad,
                        unsigned* __restrict__ hist0, int* status) {
    extern __shared__ unsigned char tc_smem_raw[];
    unsigned char* smem = reinterpret_cast<unsigned char*>(
        (reinterpret_cast<uintptr_t>(tc_smem_raw) + 1023) & ~uintptr_t(1023));
    uint64_t* full = reinterpret_cast<uint64_t*>(smem + STAGES * STAGE_BYTES);
    uint64_t* empty = full + STAGES;
    uint64_t* tfull = empty + STAGES;
    uint64_t* tempty = tfull + 2;
    uint64_t* drain = tempty + 2;
    uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(drain + 1);
    volatile int* abort_flag = reinterpret_cast<volatile int*>(tmem_slot + 1);
    float* colscale = reinterpret_cast<float*>(tmem_slot + 4);
    // first-level selection histograms of the two extreme sides (HIST_BINS
    // bins each, keys order_key(max) and order_key(-min)), flushed to hist0 at
    // the end
    unsigned* hsh = reinterpret_cast<unsigned*>(colscale + 2 * TN);

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (hist0)
        for (int i = threadIdx.x; i < 2 * HIST_BINS; i += THREADS) hsh[i] = 0u;
    if (threadIdx.x == 0) {
        for (int s = 0; s < STAGES; ++s) {
            mbar_init(&full[s], 1);
            mbar_init(&empty[s], 1);
        }
        for (int a = 0; a < 2; ++a) {
            mbar_init(&tfull[a], 1);
            mbar_init(&tempty[a], EPI / 32);
        }
        mbar_init(drain, 1);
        *abort_flag = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 1) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                         smem_u32(tmem_slot)),
                     "r"(TMEM_COLS));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = *tmem_slot;
    const int tiles = tiles_m * tiles_n;
    auto fail = [&]() {
        *abort_flag = 1;
        set_status(status, DEV_TIMEOUT);
    };

    if (warp == 0) {
        if (lane == 0) {
            int it = 0;
            bool ok = true;
            for (int t = blockIdx.x; ok && t < tiles; t += gridDim.x) {
                const int m0 = (t / tiles_n) * TM, n0 = (t % tiles_n) * TN;
                for (int kb = 0; kb < num_kb; ++kb, ++it) {
                    const int s = it % STAGES;
                    const uint32_t ph = (it / STAGES) & 1;
                    if (!mbar_wait(&empty[s], ph ^ 1, abort_flag)) {
                        fail();
                        ok = false;
                        break;
                    }
                    unsigned char* st = smem + s * STAGE_BYTES;
                    mbar_expect_tx(&full[s], STAGE_BYTES);
                    tma_load_2d(st, &tma, &full[s], kb * 128 / (FP8 ? 1 : 2), m0);
                    tma_load_2d(st + A_BYTES, &tmb, &full[s], kb * 128 / (FP8 ? 1 : 2), n0);
                }
            }
            // drain: every issued copy has landed before the CTA may exit
            for (int i = it > STAGES ? it - STAGES : 0; i < it; ++i)
                mbar_wait(&full[i % STAGES], (i / STAGES) & 1, nullptr);
        }
    } else if (warp == 1) {
        if (lane == 0) {
            int it = 0, tc = 0;
            bool ok = true;
            for (int t = blockIdx.x; ok && t < tiles; t += gridDim.x, ++tc) {
                const int acc = tc & 1;
                if (!mbar_wait(&tempty[acc], ((tc >> 1) & 1) ^ 1, abort_flag)) {
                    fail();
                    break;
                }
                tc_fence_after();
                const uint32_t d = tmem + acc * TN;
                for (int kb = 0; kb < num_kb; ++kb, ++it) {
                    const int s = it % STAGES;
                    if (!mbar_wait(&full[s], (it / STAGES) & 1, abort_flag)) {
                        fail();
                        ok = false;
                        break;
                    }
                    tc_fence_after();
                    const uint32_t a = smem_u32(smem + s * STAGE_BYTES);
#pragma unroll
                    for (int k = 0; k < 4; ++k)
                        mma<FP8>(d, sdesc(a + k * 32), sdesc(a + A_BYTES + k * 32),
                                 (kb | k) != 0);
                    mma_commit(&empty[s]);
                }
                if (ok) mma_commit(&tfull[acc]);
            }
            // drain: all issued MMAs complete before TMEM is released
            mma_commit(drain);
            mbar_wait(drain, 0, nullptr);
        }
    } else {
        // two warps per TMEM lane quadrant (a warp may access the quadrant
        // warp % 4), each reducing half of the tile's columns
        const int q = warp & 3;
        const int et = (warp - 2) * 32 + lane;
        const int half = (warp - 2) >> 2;
        // column scales, double-buffered: the next tile's are loaded while
        // this tile is reduced and stored before the tile's closing barrier
        auto col_scales = [&](int t, float (&out)[TN / EPI]) {
            const int n0 = (t % tiles_n) * TN;
#pragma unroll
            for (int u = 0; u < TN / EPI; ++u) {
                const int c = et + EPI * u;
                out[u] = t < tiles && n0 + c < nb ? inv_sb[n0 + c] : 0.f;
            }
        };
        if (SCALED) {
            float cs[TN / EPI];
            col_scales(blockIdx.x, cs);
#pragma unroll
            for (int u = 0; u < TN / EPI; ++u) colscale[et + EPI * u] = cs[u];
            asm volatile("bar.sync 1, %0;" ::"n"(EPI) : "memory");
        }
        int tc = 0;
        for (int t = blockIdx.x; t < tiles; t += gridDim.x, ++tc) {
            const int acc = tc & 1;
            const int m0 = (t / tiles_n) * TM, n0 = (t % tiles_n) * TN;
            const float* cscale = colscale + (tc & 1) * TN;
            float cs_next[TN / EPI];
            if (SCALED) col_scales(t + gridDim.x, cs_next);
            if (!mbar_wait(&tfull[acc], (tc >> 1) & 1, abort_flag)) {
                fail();
                // epilogue warps whose wait for this tile succeeded meet at the
                // tile's closing barrier: arrive there without waiting, so they
                // pass it and then stop at the next wait (the abort flag is set)
                if (SCALED) asm volatile("bar.arrive 1, %0;" ::"n"(EPI) : "memory");
                break;
            }
            tc_fence_after();
            const int64_t row = m0 + 32 * q + lane;
            const bool row_ok = row < na;
            const float rs = SCALED ? (row_ok ? inv_sa[row] : 0.f) : 1.f;
            // two 32-column chunks per TMEM round trip (both loads in flight,
            // one wait). With scales, a value is (acc x col scale) x row scale;
            // the row scale is positive and rounding is monotone, so it is
            // applied to the chunk's extremes instead of every value.
#pragma unroll 1
            for (int c2 = half * (TN / 64); c2 < (half + 1) * (TN / 64); c2 += 2) {
                uint32_t r[2][32];
#pragma unroll
                for (int h = 0; h < 2; ++h)
                    tmem_ld32_issue(tmem + (uint32_t)(acc * TN + (c2 + h) * 32) +
                                        ((uint32_t)(32 * q) << 16),
                                    r[h]);
                tmem_ld_wait();
#pragma unroll
                for (int h = 0; h < 2; ++h) {
                    const int c = c2 + h;
                    float v[32];
#pragma unroll
                    for (int j = 0; j < 32; ++j) v[j] = __uint_as_float(r[h][j]);
                    const int64_t col0 = n0 + c * 32;
                    if (SCALED) {
#pragma unroll
                        for (int j = 0; j < 32; ++j) v[j] = v[j] * cscale[c * 32 + j];
                    }
                    float mx = -CUDART_INF_F, mn = CUDART_INF_F;
                    if (row_ok && col0 + 31 < nb && (!self || col0 > row)) {
                        // every pair of the chunk counts: no per-value checks
#pragma unroll
                        for (int j = 0; j < 32; j += 2) {
                            mx = fmaxf(mx, fmaxf(v[j], v[j + 1]));
                            mn = fminf(mn, fminf(v[j], v[j + 1]));
                        }
                    } else {
#pragma unroll
                        for (int j = 0; j < 32; ++j) {
                            const int64_t col = col0 + j;
                            const bool ok = row_ok && col < nb && (!self || col > row);
                            mx = ok ? fmaxf(mx, v[j]) : mx;
                            mn = ok ? fminf(mn, v[j]) : mn;
                        }
                    }
                    if (SCALED) {  // +-inf (no pair of the chunk counts) stays as it is
                        if (mx > -CUDART_INF_F) mx = mx * rs;
                        if (mn < CUDART_INF_F) mn = mn * rs;
                    }
                    if (hist0) {  // lanes with the same bin add once
                        const unsigned b0 =
                            mx > -CUDART_INF_F ? order_key(mx) >> HIST_SHIFT : 0xffffffffu;
                        const unsigned b1 =
                            mn < CUDART_INF_F ? order_key(-mn) >> HIST_SHIFT : 0xffffffffu;
                        const unsigned g0 = __match_any_sync(0xffffffffu, b0);
                        if (b0 != 0xffffffffu && lane == __ffs(g0) - 1)
                            atomicAdd(&hsh[b0], (unsigned)__popc(g0));
                        const unsigned g1 = __match_any_sync(0xffffffffu, b1);
                        if (b1 != 0xffffffffu && lane == __ffs(g1) - 1)
                            atomicAdd(&hsh[HIST_BINS + b1], (unsigned)__popc(g1));
                    }
                    const int64_t chunk = (n0 >> 5) + c;
                    if (row < na_pad) {
                        cmax[chunk * na_pad + row] = mx;
                        cmin[chunk * na_pad + row] = mn;
                    }
                }
            }
            tc_fence_before();
            __syncwarp();
            if (lane == 0) mbar_arrive(&tempty[acc]);
            if (SCALED) {  // the other buffer was last read in the previous tile
                float* nxt = colscale + ((tc + 1) & 1) * TN;
#pragma unroll
                for (int u = 0; u < TN / EPI; ++u) nxt[et + EPI * u] = cs_next[u];
                asm volatile("bar.sync 1, %0;" ::"n"(EPI) : "memory");
            }
        }
    }
    tc_fence_before();
    __syncthreads();
    if (warp == 1) {
        tc_fence_after();
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem),
                     "r"(TMEM_COLS));
    }
    if (hist0)  // side s's bins at hist0 + 4096 s
        for (int i = threadIdx.x; i < 2 * HIST_BINS; i += THREADS)
            if (hsh[i]) atomicAdd(&hist0[(i / HIST_BINS) * 4096 + i % HIST_BINS], hsh[i]);
}

constexpr size_t smem_bytes() {
    return 1024 + STAGES * STAGE_BYTES + 256 + 16 + 2 * TN * 4 + 2 * HIST_BINS * 4;
}

}  // namespace tc

typedef CUresult (*EncodeTiledFn)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*,
                                   const cuuint64_t*, const cuuint64_t*, const cuuint32_t*,
                                   const cuuint32_t*, CUtensorMapInterleave, CUtensorMapSwizzle,
                                   CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

static cudaError_t make_map(CUtensorMap* m, const void* base, bool fp8, int64_t rows,
                            int64_t kbytes, int box_rows) {
    static EncodeTiledFn fn = nullptr;
    if (!fn) {
        cudaDriverEntryPointQueryResult q;
        void* p = nullptr;
        cudaError_t e = cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000,
                                                         cudaEnableDefault, &q);
        if (e != cudaSuccess || q != cudaDriverEntryPointSuccess || !p)
            return e != cudaSuccess ? e : cudaErrorNotSupported;
        fn = reinterpret_cast<EncodeTiledFn>(p);
    }
    const int esz = fp8 ? 1 : 2;
    cuuint64_t gdim[2] = {(cuuint64_t)(kbytes / esz), (cuuint64_t)rows};
    cuuint64_t gstride[1] = {(cuuint64_t)kbytes};
    cuuint32_t box[2] = {(cuuint32_t)(128 / esz), (cuuint32_t)box_rows};
    cuuint32_t estride[2] = {1, 1};
    CUresult r = fn(m, fp8 ? CU_TENSOR_MAP_DATA_TYPE_UINT8 : CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2,
                    const_cast<void*>(base), gdim, gstride, box, estride,
                    CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B,
                    CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    return r == CUDA_SUCCESS ? cudaSuccess : cudaErrorInvalidValue;
}

// qa: [na_pad][kbytes] operand A (rows padded to 256), qb likewise; kbytes a
// multiple of 128. Writes cmax/cmin [nb_pad/32][na_pad]; with hist0, also
// adds the first-level selection histograms of both sides (bins of the top 11
// key bits; side s at hist0 + 4096 s, which the caller zeroes).
cudaError_t launch_tc_chunk_extremes(bool fp8, bool scaled, const void* qa, int64_t na, int64_t na_pad,
                                     const void* qb, int64_t nb, int64_t nb_pad, int64_t kbytes,
                                     int self, const float* inv_sa, const float* inv_sb,
                                     float* cmax, float* cmin, unsigned* hist0, int* status,
                                     cudaStream_t st) {
    if (kbytes % 128 || na_pad % 256 || nb_pad % 256) return cudaErrorInvalidValue;
    CUtensorMap ma, mb;
    cudaError_t e = make_map(&ma, qa, fp8, na_pad, kbytes, tc::TM);
    if (e == cudaSuccess) e = make_map(&mb, qb, fp8, nb_pad, kbytes, tc::TN);
    if (e != cudaSuccess) return e;
    // every padded row is covered (rows past na hold -inf / +inf), so the
    // selection passes never read an extreme this call did not write
    const int tiles_m = (int)(na_pad / tc::TM);
    const int tiles_n = (int)((nb + tc::TN - 1) / tc::TN);
    int dev = 0, sms = 148;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    const int tiles = tiles_m * tiles_n;
    const int grid = tiles < sms ? tiles : sms;
    const size_t smem = tc::smem_bytes();
    if (fp8 && !scaled) return cudaErrorInvalidValue;  // FP8 operands always carry scales
    auto kern = fp8      ? tc::k_tc_chunk_extremes<true, true>
                : scaled ? tc::k_tc_chunk_extremes<false, true>
                         : tc::k_tc_chunk_extremes<false, false>;
    e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    note_launch();
    kern<<<grid, tc::THREADS, smem, st>>>(ma, mb, (int)(kbytes / 128), na, nb, tiles_m, tiles_n,
                                          self, inv_sa, inv_sb, cmax, cmin, na_pad, hist0,
                                          status);
    return cudaGetLastError();
}

}  // namespace cc
