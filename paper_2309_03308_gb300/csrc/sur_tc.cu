// All-pairs screen of the learned surrogate on the 5th-generation tensor
// cores (project addition; the paper's Section 7 names a network predicting
// MI as future work). For region points a and b the head's first layer is
//   z = W3 [e_a, e_b, |e_a - e_b|, off] + b3
//     = (Wa e_a + b3) + [Wc, Wb] [|e_a - e_b| ; e_b] + Wd off,
// with Wa e_a + b3 computed once per point. A tile is one point a and 128
// points b: the 128 x 128 operand [|e_a - e_b|, e_b] (BF16, written into
// shared memory in the 128-byte-swizzled K-major layout by the producer
// warps) times [Wc, Wb]^T (128 hidden x 128, BF16, loaded once per CTA)
// accumulates in TMEM (FP32). The epilogue adds Wa e_a + b3 and Wd off,
// applies GELU (erf form) and the output layer y = w4 . h + b4, and stores the
// de-standardized prediction. Self region pairs get -inf for b <= a.
//
// Warp roles (416 threads, one CTA per SM, persistent over tiles):
//   warps 0-3   producers: one pair row each per thread, 3-stage ring
//   warp 4      TMEM allocation + MMA issuer (8 MMAs of K = 16 per tile)
//   warps 5-12  epilogue in two groups of four that take alternate tiles
//               (and accumulators); warp w reads TMEM lanes 32 (w % 4) .. +31
// Every mbarrier wait is bounded; on timeout the CTA records DEV_TIMEOUT, the
// other roles leave their loops, MMAs are drained and TMEM is freed.
#include <cuda_bf16.h>

#include "device.cuh"
#include "internal.cuh"
#include "tc_dev.cuh"

namespace cc {
namespace tc {

constexpr int SC_ROWS = 128;                    // pairs per tile (MMA M)
constexpr int SC_N = 128;                       // hidden units (MMA N)
constexpr int SC_E = 64;                        // embedding width
constexpr int SC_HEAD_IN = 3 * SC_E + 3;        // W3 row length
constexpr int SC_ATOM = SC_ROWS * 128;          // one 64-element K atom of 128 rows, 16 KB
constexpr int SC_A_BYTES = 2 * SC_ATOM;         // [|e_a - e_b| atom, e_b atom]
constexpr int SC_B_BYTES = 2 * SC_N * 128;      // [Wc atom, Wb atom]
constexpr int SC_STAGES = 3;
constexpr int SC_PROD = 128, SC_EPI_WARPS = 8;
constexpr int SC_THREADS = SC_PROD + 32 + 32 * SC_EPI_WARPS;  // 416
constexpr int SC_TMEM_COLS = 2 * SC_N;                        // two accumulators

__host__ __device__ constexpr uint32_t sc_idesc() {  // FP32 acc, BF16 x BF16, K-major, N, M
    return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(SC_N >> 3) << 17) |
           ((uint32_t)(SC_ROWS >> 4) << 24);
}
__device__ __forceinline__ void sc_mma(uint32_t d, uint64_t a, uint64_t b, uint32_t accum) {
    asm volatile(
        "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(d),
        "l"(a), "l"(b), "r"(sc_idesc()), "r"(accum));
}
// byte offset of the 16-byte chunk c (elements 8c .. 8c+7) of row r in a
// K-major, 128-byte-swizzled atom (rows of 128 bytes, 8-row groups of 1024)
__device__ __forceinline__ uint32_t sw128(int r, int c) {
    return (uint32_t)(r * 128 + ((c ^ (r & 7)) << 4));
}
__device__ __forceinline__ uint32_t pack_bf16x2(float lo, float hi) {
    const __nv_bfloat162 v = __floats2bfloat162_rn(lo, hi);
    return *reinterpret_cast<const uint32_t*>(&v);
}
__device__ __forceinline__ float sc_gelu(float x) {
    return 0.5f * x * (1.f + erff(x * 0.70710678118654752f));
}

__global__ void __launch_bounds__(SC_THREADS, 1)
    k_sur_screen_tc(const float* __restrict__ Ea, const float* __restrict__ Ua,
                    const float* __restrict__ Eb, const __nv_bfloat16* __restrict__ wb,
                    const float* __restrict__ w, int64_t oW3, int64_t ow4, int64_t ob4,
                    const uint32_t* __restrict__ pts_a, const uint32_t* __restrict__ pts_b,
                    int64_t na, int64_t nb, int self, int X, int Y, int Z, float tmean,
                    float tsd, float* __restrict__ pred, int* status) {
    extern __shared__ unsigned char sc_smem_raw[];
    unsigned char* smem = reinterpret_cast<unsigned char*>(
        (reinterpret_cast<uintptr_t>(sc_smem_raw) + 1023) & ~uintptr_t(1023));
    unsigned char* Bt = smem;                           // SC_B_BYTES
    unsigned char* At = Bt + SC_B_BYTES;                // SC_STAGES x SC_A_BYTES
    float* wd = reinterpret_cast<float*>(At + SC_STAGES * SC_A_BYTES);  // [128][3]
    float* w4 = wd + 3 * SC_N;                                           // [128]
    uint64_t* full = reinterpret_cast<uint64_t*>(w4 + SC_N);
    uint64_t* empty = full + SC_STAGES;
    uint64_t* tfull = empty + SC_STAGES;
    uint64_t* tempty = tfull + 2;
    uint64_t* drain = tempty + 2;
    uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(drain + 1);
    volatile int* abort_flag = reinterpret_cast<volatile int*>(tmem_slot + 1);

    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    // weights: [Wc, Wb] as the B operand (BF16, swizzled), Wd and w4 (fp32)
    for (int e = tid; e < 2 * SC_N * 8; e += blockDim.x) {
        const int atom = e / (SC_N * 8), h = (e / 8) % SC_N, c = e % 8;
        // W3 rows are 195 elements long: read element-wise (no 16-byte alignment)
        const unsigned short* src = reinterpret_cast<const unsigned short*>(wb) + oW3 +
                                    (int64_t)h * SC_HEAD_IN + (atom == 0 ? 2 * SC_E : SC_E) +
                                    8 * c;
        uint32_t u[4];
#pragma unroll
        for (int j = 0; j < 4; ++j) u[j] = (uint32_t)src[2 * j] | ((uint32_t)src[2 * j + 1] << 16);
        *reinterpret_cast<uint4*>(Bt + atom * (SC_N * 128) + sw128(h, c)) =
            make_uint4(u[0], u[1], u[2], u[3]);
    }
    for (int e = tid; e < 3 * SC_N; e += blockDim.x)
        wd[e] = w[oW3 + (int64_t)(e / 3) * SC_HEAD_IN + 3 * SC_E + e % 3];
    for (int e = tid; e < SC_N; e += blockDim.x) w4[e] = w[ow4 + e];
    if (tid == 0) {
        for (int s = 0; s < SC_STAGES; ++s) {
            mbar_init(&full[s], SC_PROD);
            mbar_init(&empty[s], 1);
        }
        for (int a = 0; a < 2; ++a) {
            mbar_init(&tfull[a], 1);
            mbar_init(&tempty[a], SC_EPI_WARPS / 2);
        }
        mbar_init(drain, 1);
        *abort_flag = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 4) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                         smem_u32(tmem_slot)),
                     "r"(SC_TMEM_COLS));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
    }
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");  // B operand -> tensor core
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = *tmem_slot;
    const int64_t nbt = (nb + SC_ROWS - 1) / SC_ROWS;
    const int64_t tiles = na * nbt;
    const float b4 = w[ob4];
    auto fail = [&]() {
        *abort_flag = 1;
        set_status(status, DEV_TIMEOUT);
    };

    if (warp < 4) {  // producers: row r = tid of every tile
        const int r = tid;
        int it = 0;
        for (int64_t t = blockIdx.x; t < tiles; t += gridDim.x, ++it) {
            const int s = it % SC_STAGES;
            if (!mbar_wait(&empty[s], ((it / SC_STAGES) & 1) ^ 1, abort_flag)) {
                fail();
                break;
            }
            const int64_t a = t / nbt, b = (t % nbt) * SC_ROWS + r;
            const float4* ea = reinterpret_cast<const float4*>(Ea + a * SC_E);
            const float4* eb = reinterpret_cast<const float4*>(Eb + (b < nb ? b : 0) * SC_E);
            unsigned char* st = At + s * SC_A_BYTES;
#pragma unroll
            for (int c = 0; c < 8; ++c) {
                const float4 x0 = ea[2 * c], x1 = ea[2 * c + 1];
                float4 y0 = eb[2 * c], y1 = eb[2 * c + 1];
                if (b >= nb) y0 = y1 = make_float4(0.f, 0.f, 0.f, 0.f);
                const uint4 dv = make_uint4(
                    pack_bf16x2(fabsf(x0.x - y0.x), fabsf(x0.y - y0.y)),
                    pack_bf16x2(fabsf(x0.z - y0.z), fabsf(x0.w - y0.w)),
                    pack_bf16x2(fabsf(x1.x - y1.x), fabsf(x1.y - y1.y)),
                    pack_bf16x2(fabsf(x1.z - y1.z), fabsf(x1.w - y1.w)));
                const uint4 bv = make_uint4(pack_bf16x2(y0.x, y0.y), pack_bf16x2(y0.z, y0.w),
                                            pack_bf16x2(y1.x, y1.y), pack_bf16x2(y1.z, y1.w));
                *reinterpret_cast<uint4*>(st + sw128(r, c)) = dv;
                *reinterpret_cast<uint4*>(st + SC_ATOM + sw128(r, c)) = bv;
            }
            asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
            mbar_arrive(&full[s]);
        }
    } else if (warp == 4) {  // MMA issuer
        if (lane == 0) {
            int it = 0;
            bool ok = true;
            const uint32_t bA = smem_u32(At), bB = smem_u32(Bt);
            for (int64_t t = blockIdx.x; ok && t < tiles; t += gridDim.x, ++it) {
                const int acc = it & 1, s = it % SC_STAGES;
                if (!mbar_wait(&tempty[acc], ((it >> 1) & 1) ^ 1, abort_flag) ||
                    !mbar_wait(&full[s], (it / SC_STAGES) & 1, abort_flag)) {
                    fail();
                    ok = false;
                    break;
                }
                tc_fence_after();
                const uint32_t d = tmem + acc * SC_N;
                const uint32_t a0 = bA + s * SC_A_BYTES;
#pragma unroll
                for (int atom = 0; atom < 2; ++atom)
#pragma unroll
                    for (int k = 0; k < 4; ++k)
                        sc_mma(d, sdesc(a0 + atom * SC_ATOM + k * 32),
                               sdesc(bB + atom * (SC_N * 128) + k * 32), (atom | k) != 0);
                mma_commit(&empty[s]);
                mma_commit(&tfull[acc]);
            }
            mma_commit(drain);  // every issued MMA completes before TMEM is released
            mbar_wait(drain, 0, nullptr);
        }
    } else {  // epilogue: group g = (warp - 5) / 4 takes the tiles with it % 2 == g
        const int q = warp & 3, g = (warp - 5) >> 2;
        const int r = 32 * q + lane;
        int it = 0;
        for (int64_t t = blockIdx.x; t < tiles; t += gridDim.x, ++it) {
            if ((it & 1) != g) continue;
            const int acc = g;
            if (!mbar_wait(&tfull[acc], (it >> 1) & 1, abort_flag)) {
                fail();
                break;
            }
            tc_fence_after();
            const int64_t a = t / nbt, b = (t % nbt) * SC_ROWS + r;
            const bool live = b < nb;
            float o0 = 0.f, o1 = 0.f, o2 = 0.f;
            if (live) {
                const int64_t p = pts_a[a], qq = pts_b[b];
                o0 = (float)((qq % X) - (p % X)) / (float)X;
                o1 = (float)(((qq / X) % Y) - ((p / X) % Y)) / (float)Y;
                o2 = (float)((qq / ((int64_t)X * Y)) - (p / ((int64_t)X * Y))) / (float)Z;
            }
            const float* ua = Ua + a * SC_N;
            float y = 0.f;
            const uint32_t base = tmem + ((uint32_t)(32 * q) << 16) + acc * SC_N;
#pragma unroll 1
            for (int c0 = 0; c0 < SC_N; c0 += 32) {
                float v[32];
                tmem_ld32(base + c0, v);
                if (c0 + 32 == SC_N) {  // last columns read: release the accumulator
                    tc_fence_before();
                    __syncwarp();
                    if (lane == 0) mbar_arrive(&tempty[acc]);
                }
#pragma unroll
                for (int i = 0; i < 32; ++i) {
                    const int h = c0 + i;
                    float z = v[i] + ua[h];
                    z = fmaf(wd[3 * h + 0], o0, z);
                    z = fmaf(wd[3 * h + 1], o1, z);
                    z = fmaf(wd[3 * h + 2], o2, z);
                    y = fmaf(w4[h], sc_gelu(z), y);
                }
            }
            if (live) {
                float out = (y + b4) * tsd + tmean;
                if (self && b <= a) out = -CUDART_INF_F;  // each unordered pair once
                pred[a * nb + b] = out;
            }
        }
    }
    tc_fence_before();
    __syncthreads();
    if (warp == 4) {
        tc_fence_after();
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem),
                     "r"(SC_TMEM_COLS));
    }
}

constexpr size_t sc_smem_bytes() {
    return 1024 + SC_B_BYTES + SC_STAGES * SC_A_BYTES + 4 * (3 * SC_N + SC_N) +
           8 * (2 * SC_STAGES + 5) + 16;
}

}  // namespace tc

// Predictions for all pairs of two regions: Ea/Eb [n][64] embeddings, Ua
// [na][128] = Wa e_a + b3 (fp32), wb / w the BF16 and fp32 parameter vectors.
cudaError_t launch_sur_screen_tc(const float* Ea, const float* Ua, const float* Eb,
                                 const void* wb, const float* w, int64_t oW3, int64_t ow4,
                                 int64_t ob4, const uint32_t* pts_a, const uint32_t* pts_b,
                                 int64_t na, int64_t nb, int self, int X, int Y, int Z,
                                 float tmean, float tsd, float* pred, int* status,
                                 cudaStream_t st) {
    if (na < 1 || nb < 1) return cudaErrorInvalidValue;
    const size_t smem = tc::sc_smem_bytes();
    cudaError_t e = cudaFuncSetAttribute(tc::k_sur_screen_tc,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    int dev = 0, sms = 148;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    const int64_t tiles = na * ((nb + tc::SC_ROWS - 1) / tc::SC_ROWS);
    const int grid = (int)(tiles < sms ? tiles : sms);
    note_launch();
    tc::k_sur_screen_tc<<<grid, tc::SC_THREADS, smem, st>>>(
        Ea, Ua, Eb, reinterpret_cast<const __nv_bfloat16*>(wb), w, oW3, ow4, ob4, pts_a, pts_b,
        na, nb, self, X, Y, Z, tmean, tsd, pred, status);
    return cudaGetLastError();
}

}  // namespace cc
