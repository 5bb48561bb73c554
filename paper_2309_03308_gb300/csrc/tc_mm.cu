// General matrix product on the 5th-generation tensor cores, used by the
// learned surrogate's training step (project addition; the paper's Section 7
// names a network predicting MI as future work):
//
//   C[m][n] (+)= sum_k A(m, k) B(n, k),  A(m, k) = A[m sam + k sak],
//                                        B(n, k) = B[n sbn + k sbk]
//
// with each operand BF16 or FP32 in memory and any pair of strides, so one
// kernel serves the forward layers (activations times weights), the data
// gradients (gradients times weights read along their output dimension) and
// the weight gradients (gradients and activations both read across the
// batch). FP32 operands are rounded to BF16 when they are staged; products
// accumulate in FP32 in TMEM.
//
// A CTA owns 128 rows of C (the MMA's M) and all N <= 256 columns (N rounded
// up to 16 is the MMA's N); K advances 64 at a time through a 4-stage ring of
// shared-memory tiles in the K-major, 128-byte-swizzled layout (rows of 128
// bytes, 8-row groups 1024 bytes apart). Rows past M or N and k past the end
// are staged as zeros. Split-K: grid z slices K into chunks of kc and each
// slice writes a dense FP32 partial [z][M][N] (summed in slice order by the
// caller, so results do not depend on timing).
//
// Warp roles (256 threads): warps 0-6 stage both operands (16-byte reads of
// chunks along k when the source is contiguous along k, of eight-row groups
// when it is contiguous along rows; element reads at unaligned strides and
// ragged edges), then warps 0-3 read the accumulator back (warp q owns TMEM
// lanes 32q .. 32q + 31, i.e. the tile's rows) and store it in row segments of
// 32 columns transposed through shared memory; warp 7 allocates
// TMEM and one of its threads issues the MMAs (4 of K = 16 per stage). Every
// mbarrier wait is bounded; on timeout the CTA records DEV_TIMEOUT, the roles
// leave their loops, issued MMAs are drained and TMEM is freed.
#include <cuda_bf16.h>

#include "device.cuh"
#include "internal.cuh"
#include "tc_dev.cuh"

namespace cc {
namespace tc {

constexpr int MM_M = 128;                 // rows of C per CTA (MMA M)
constexpr int MM_STAGES = 4;
constexpr int MM_A_BYTES = MM_M * 128;    // 128 rows x 64 BF16
constexpr int MM_PROD = 224;            // staging threads (warps 0-6)
constexpr int MM_THREADS = MM_PROD + 32;
constexpr int MM_MAX_N = 256;

struct MmOp {
    const void* p;
    int64_t s_row, s_k;  // element (row, k) at p[row s_row + k s_k]
    int bf16;            // element type: BF16 (1) or FP32 (0)
    int64_t ones;        // a row that reads as 1 for every k (-1: none; rows mode only)
};

template <int MODE>
__device__ __forceinline__ float mm_ld(const MmOp& o, int64_t i) {
    if constexpr ((MODE & 2) != 0)
        return __bfloat162float(reinterpret_cast<const __nv_bfloat16*>(o.p)[i]);
    else
        return reinterpret_cast<const float*>(o.p)[i];
}
__device__ __forceinline__ uint32_t mm_pack(float lo, float hi) {
    return (uint32_t)__bfloat16_as_ushort(__float2bfloat16_rn(lo)) |
           ((uint32_t)__bfloat16_as_ushort(__float2bfloat16_rn(hi)) << 16);
}
__host__ __device__ constexpr uint32_t mm_idesc(int np) {  // FP32 acc, BF16 x BF16, K-major
    return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(np >> 3) << 17) |
           ((uint32_t)(MM_M >> 4) << 24);
}
__device__ __forceinline__ void mm_mma(uint32_t d, uint64_t a, uint64_t b, uint32_t idesc,
                                       uint32_t accum) {
    asm volatile(
        "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(d),
        "l"(a), "l"(b), "r"(idesc), "r"(accum));
}

// Staging of rows [r0, r0 + rows) x k in [k0, k0 + 64) of an operand as BF16
// into a swizzled tile (chunk c of row r, elements 8c .. 8c + 7, at sw(r, c));
// rows >= nrows and k >= ke are zero; rows is a multiple of 16, at most 256.
// Two unit shapes:
//   along k (s_k == 1): unit = (row r, chunk c), consecutive threads take
//     consecutive chunks of a row; one 16-byte read when vec;
//   along rows (otherwise): unit = (eight-row group g, k pair kp),
//     consecutive threads take consecutive k pairs of one group (their
//     shared-memory words then fall in distinct banks); two 16-byte reads
//     (BF16) or four (FP32) of eight consecutive rows when vec, and the
//     thread writes one BF16 pair into each of the eight rows. A row equal
//     to o.ones reads as 1 (a column sum rides along as one more output).
// vec: the operand's base and its stride across the contiguous dimension are
// 16-byte aligned; ragged units fall back to element reads. A thread first
// reads all of its units of both operands into registers and only then
// writes shared memory, so a stage costs one round of memory latency.
__device__ __forceinline__ uint32_t mm_sw(int r, int c) {
    return (uint32_t)(r * 128 + ((c ^ (r & 7)) << 4));
}
constexpr int MM_UMAX = (256 * 8 + MM_PROD - 1) / MM_PROD;  // units per thread, at most

struct MmUnits {
    uint32_t w[MM_UMAX][4];
};

// operand modes: contiguous along k or along rows, BF16 or FP32
constexpr int MM_ALONG_K = 1, MM_BF16 = 2;

template <int MODE>
__device__ __forceinline__ void mm_load(MmUnits& U, const MmOp& o, int64_t r0, int rows,
                                        int64_t nrows, int64_t k0, int64_t ke, int t) {
    constexpr bool vec = true;
    if constexpr ((MODE & MM_ALONG_K) != 0) {
#pragma unroll
        for (int i = 0; i < MM_UMAX; ++i) {
            const int u = t + i * MM_PROD;
            U.w[i][0] = U.w[i][1] = U.w[i][2] = U.w[i][3] = 0u;
            if (u >= rows * 8) continue;
            const int r = u >> 3, c = u & 7;
            const int64_t row = r0 + r, k = k0 + 8 * c;
            if (row >= nrows) continue;
            const int64_t base = row * o.s_row + k;
            if (vec && k + 8 <= ke) {
                if constexpr ((MODE & MM_BF16) != 0) {
                    const uint4 x = *reinterpret_cast<const uint4*>(
                        reinterpret_cast<const __nv_bfloat16*>(o.p) + base);
                    U.w[i][0] = x.x;
                    U.w[i][1] = x.y;
                    U.w[i][2] = x.z;
                    U.w[i][3] = x.w;
                } else {
                    const float4* f =
                        reinterpret_cast<const float4*>(reinterpret_cast<const float*>(o.p) + base);
                    const float4 a = f[0], b = f[1];
                    U.w[i][0] = mm_pack(a.x, a.y);
                    U.w[i][1] = mm_pack(a.z, a.w);
                    U.w[i][2] = mm_pack(b.x, b.y);
                    U.w[i][3] = mm_pack(b.z, b.w);
                }
            } else {
#pragma unroll
                for (int j = 0; j < 4; ++j) {
                    const float v0 = k + 2 * j < ke ? mm_ld<MODE>(o, base + 2 * j) : 0.f;
                    const float v1 = k + 2 * j + 1 < ke ? mm_ld<MODE>(o, base + 2 * j + 1) : 0.f;
                    U.w[i][j] = mm_pack(v0, v1);
                }
            }
        }
    } else {
        // a unit here carries eight pairs; two units' worth of registers per slot
        const int groups = rows >> 3;
#pragma unroll
        for (int i = 0; i < MM_UMAX / 2; ++i) {
            const int u = t + i * MM_PROD;
            uint32_t* w = &U.w[2 * i][0];  // 8 words: rows 8g .. 8g + 7
#pragma unroll
            for (int j = 0; j < 8; ++j) w[j] = 0u;
            if (u >= groups * 32) continue;
            const int kp = u & 31, g = u >> 5;
            const int64_t row = r0 + 8 * g, k = k0 + 2 * kp;
            if (vec && row + 8 <= nrows && k + 2 <= ke && (o.ones < row || o.ones >= row + 8)) {
                const int64_t b0 = row + k * o.s_k, b1 = b0 + o.s_k;
                if constexpr ((MODE & MM_BF16) != 0) {
                    const __nv_bfloat16* q = reinterpret_cast<const __nv_bfloat16*>(o.p);
                    const uint4 x = *reinterpret_cast<const uint4*>(q + b0);
                    const uint4 y = *reinterpret_cast<const uint4*>(q + b1);
                    const uint32_t xw[4] = {x.x, x.y, x.z, x.w}, yw[4] = {y.x, y.y, y.z, y.w};
#pragma unroll
                    for (int j = 0; j < 4; ++j) {  // row pair j: (k, k + 1) of rows 2j, 2j + 1
                        w[2 * j] = (xw[j] & 0xffffu) | (yw[j] << 16);
                        w[2 * j + 1] = (xw[j] >> 16) | (yw[j] & 0xffff0000u);
                    }
                } else {
                    const float* q = reinterpret_cast<const float*>(o.p);
                    const float4 a0 = *reinterpret_cast<const float4*>(q + b0);
                    const float4 a1 = *reinterpret_cast<const float4*>(q + b0 + 4);
                    const float4 c0 = *reinterpret_cast<const float4*>(q + b1);
                    const float4 c1 = *reinterpret_cast<const float4*>(q + b1 + 4);
                    w[0] = mm_pack(a0.x, c0.x);
                    w[1] = mm_pack(a0.y, c0.y);
                    w[2] = mm_pack(a0.z, c0.z);
                    w[3] = mm_pack(a0.w, c0.w);
                    w[4] = mm_pack(a1.x, c1.x);
                    w[5] = mm_pack(a1.y, c1.y);
                    w[6] = mm_pack(a1.z, c1.z);
                    w[7] = mm_pack(a1.w, c1.w);
                }
            } else {
#pragma unroll
                for (int j = 0; j < 8; ++j) {
                    const bool ok = row + j < nrows, one = row + j == o.ones;
                    const int64_t b = (row + j) * o.s_row + k * o.s_k;
                    const float v0 = ok && k < ke ? (one ? 1.f : mm_ld<MODE>(o, b)) : 0.f;
                    const float v1 = ok && k + 1 < ke ? (one ? 1.f : mm_ld<MODE>(o, b + o.s_k)) : 0.f;
                    w[j] = mm_pack(v0, v1);
                }
            }
        }
    }
}

template <int MODE>
__device__ __forceinline__ void mm_store(unsigned char* dst, const MmUnits& U, int rows, int t) {
    if constexpr ((MODE & MM_ALONG_K) != 0) {
#pragma unroll
        for (int i = 0; i < MM_UMAX; ++i) {
            const int u = t + i * MM_PROD;
            if (u < rows * 8)
                *reinterpret_cast<uint4*>(dst + mm_sw(u >> 3, u & 7)) =
                    make_uint4(U.w[i][0], U.w[i][1], U.w[i][2], U.w[i][3]);
        }
    } else {
        const int groups = rows >> 3;
#pragma unroll
        for (int i = 0; i < MM_UMAX / 2; ++i) {
            const int u = t + i * MM_PROD;
            if (u >= groups * 32) continue;
            const int kp = u & 31, g = u >> 5;
            const uint32_t* w = &U.w[2 * i][0];
#pragma unroll
            for (int j = 0; j < 8; ++j)
                *reinterpret_cast<uint32_t*>(dst + mm_sw(8 * g + j, kp >> 2) + (kp & 3) * 4) =
                    w[j];
        }
    }
}

template <int AM, int BM>
__global__ void __launch_bounds__(MM_THREADS, 1)
    k_tc_mm(MmOp A_, MmOp B_, float* __restrict__ C, int64_t ldc, int M, int N, int np, int64_t K,
            int64_t kc, float* __restrict__ part, int* status) {
    const MmOp A{A_.p, A_.s_row, A_.s_k, A_.bf16, A_.ones}, B{B_.p, B_.s_row, B_.s_k, B_.bf16, B_.ones};
    extern __shared__ unsigned char mm_smem_raw[];
    unsigned char* smem = reinterpret_cast<unsigned char*>(
        (reinterpret_cast<uintptr_t>(mm_smem_raw) + 1023) & ~uintptr_t(1023));
    const int b_bytes = np * 128;
    unsigned char* At = smem;                         // MM_STAGES x MM_A_BYTES
    unsigned char* Bt = At + MM_STAGES * MM_A_BYTES;  // MM_STAGES x b_bytes
    uint64_t* full = reinterpret_cast<uint64_t*>(Bt + MM_STAGES * b_bytes);
    uint64_t* empty = full + MM_STAGES;
    uint64_t* done = empty + MM_STAGES;
    uint64_t* drain = done + 1;
    uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(drain + 1);
    volatile int* abort_flag = reinterpret_cast<volatile int*>(tmem_slot + 1);

    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int64_t m0 = (int64_t)blockIdx.x * MM_M;
    const int64_t kb = (int64_t)blockIdx.z * kc, ke = min(K, kb + kc);
    const int nk = (int)((ke - kb + 63) / 64);
    const uint32_t tcols = np <= 32 ? 32u : (np <= 64 ? 64u : (np <= 128 ? 128u : 256u));
    if (tid == 0) {
        for (int s = 0; s < MM_STAGES; ++s) {
            mbar_init(&full[s], MM_PROD);
            mbar_init(&empty[s], 1);
        }
        mbar_init(done, 1);
        mbar_init(drain, 1);
        *abort_flag = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 7) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                         smem_u32(tmem_slot)),
                     "r"(tcols));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = *tmem_slot;
    auto fail = [&]() {
        *abort_flag = 1;
        set_status(status, DEV_TIMEOUT);
    };

    if (warp < 7) {
        bool ok = true;
        for (int it = 0; it < nk; ++it) {
            const int s = it % MM_STAGES;
            if (it >= MM_STAGES &&
                !mbar_wait(&empty[s], ((it / MM_STAGES) & 1) ^ 1, abort_flag)) {
                fail();
                ok = false;
                break;
            }
            const int64_t k0 = kb + (int64_t)it * 64;
            MmUnits ua, ub;
            mm_load<AM>(ua, A, m0, MM_M, M, k0, ke, tid);
            mm_load<BM>(ub, B, 0, np, N, k0, ke, tid);
            mm_store<AM>(At + s * MM_A_BYTES, ua, MM_M, tid);
            mm_store<BM>(Bt + s * b_bytes, ub, np, tid);
            asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
            mbar_arrive(&full[s]);
        }
        if (warp < 4) {  // epilogue: TMEM lane r = this thread's row of the tile
            if (ok && !mbar_wait(done, 0, abort_flag)) {
                fail();
                ok = false;
            }
            if (ok) {
                // 32 x 32 blocks through shared memory (the consumed stage-0 A
                // tile; XOR-swizzled, conflict-free): lane = row on the way in,
                // lane = column on the way out, so each store instruction writes
                // 32 consecutive floats of one row
                tc_fence_after();
                float* T = reinterpret_cast<float*>(At) + warp * 1024;
                const uint32_t base = tmem + ((uint32_t)(32 * warp) << 16);
                const int64_t rbase = m0 + 32 * warp;
#pragma unroll 1
                for (int c0 = 0; c0 < np; c0 += 32) {
                    float v[32];
                    tmem_ld32(base + c0, v);
#pragma unroll
                    for (int i = 0; i < 32; ++i) T[lane * 32 + (i ^ lane)] = v[i];
                    __syncwarp();
                    const int n = c0 + lane;
#pragma unroll 4
                    for (int j = 0; j < 32; ++j) {
                        const int64_t m = rbase + j;
                        if (m < M && n < N) {
                            float* out =
                                part ? part + ((int64_t)blockIdx.z * M + m) * ldc : C + m * ldc;
                            out[n] = T[j * 32 + (lane ^ j)];
                        }
                    }
                    __syncwarp();
                }
            }
        }
    } else if (lane == 0) {  // warp 7: MMA issuer
        const uint32_t idesc = mm_idesc(np);
        const uint32_t bA = smem_u32(At), bB = smem_u32(Bt);
        bool ok = true;
        for (int it = 0; it < nk; ++it) {
            const int s = it % MM_STAGES;
            if (!mbar_wait(&full[s], (it / MM_STAGES) & 1, abort_flag)) {
                fail();
                ok = false;
                break;
            }
            tc_fence_after();
#pragma unroll
            for (int k = 0; k < 4; ++k)
                mm_mma(tmem, sdesc(bA + s * MM_A_BYTES + k * 32), sdesc(bB + s * b_bytes + k * 32),
                       idesc, (it | k) != 0);
            mma_commit(&empty[s]);
        }
        if (ok) mma_commit(done);
        mma_commit(drain);  // every issued MMA completes before TMEM is released
        mbar_wait(drain, 0, nullptr);
    }
    tc_fence_before();
    __syncthreads();
    if (warp == 7) {
        tc_fence_after();
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem),
                     "r"(tcols));
    }
}

inline size_t mm_smem_bytes(int np) {
    return 1024 + (size_t)MM_STAGES * (MM_A_BYTES + (size_t)np * 128) + 8 * (2 * MM_STAGES + 2) +
           16;
}

// the operand's mode, or -1 when it is not contiguous along k or rows with a
// 16-byte aligned base and stride
inline int mm_mode(const void* p, int64_t s_row, int64_t s_k, int bf16) {
    const int64_t elt = bf16 ? 2 : 4;
    if ((reinterpret_cast<uintptr_t>(p) & 15) != 0) return -1;
    if (s_k == 1) return (s_row * elt) % 16 == 0 ? (MM_ALONG_K | (bf16 ? MM_BF16 : 0)) : -1;
    if (s_row == 1) return (s_k * elt) % 16 == 0 ? (bf16 ? MM_BF16 : 0) : -1;
    return -1;
}

}  // namespace tc

// C[m][n] = sum_k A(m, k) B(n, k) (see the top of this file). With part
// given, the z-th K slice of kc (a multiple of 64) writes part[z][M][ldc]
// instead (required when kc < K).
// b_ones >= 0: B's row b_ones reads as 1 for every k (B contiguous along rows
// only), so C's column b_ones holds the row sums of A over k.
// Returns cudaErrorNotSupported (nothing queued) when an operand is not
// contiguous along k or rows with 16-byte aligned base and stride, or when
// the pair of operand layouts has no instantiation: the caller then uses the
// SIMT product.
cudaError_t launch_tc_mm(const void* A, int a_bf16, int64_t sam, int64_t sak, const void* B,
                         int b_bf16, int64_t sbn, int64_t sbk, int64_t b_ones, float* C,
                         int64_t ldc, int M, int N, int64_t K, int64_t kc, float* part,
                         int* status, cudaStream_t st) {
    if (M < 1 || N < 1 || N > tc::MM_MAX_N || K < 1 || kc < 64 || kc % 64 != 0 || ldc < N)
        return cudaErrorInvalidValue;
    const int am = tc::mm_mode(A, sam, sak, a_bf16), bm = tc::mm_mode(B, sbn, sbk, b_bf16);
    using namespace tc;
    // the instantiated pairs: forward (activations x weights), data gradients
    // (FP32 gradients x weights along their rows), weight gradients (FP32
    // gradients x activations, both across the batch)
    void (*kern)(MmOp, MmOp, float*, int64_t, int, int, int, int64_t, int64_t, float*, int*) =
        nullptr;
    if (am == (MM_ALONG_K | MM_BF16) && bm == (MM_ALONG_K | MM_BF16))
        kern = k_tc_mm<MM_ALONG_K | MM_BF16, MM_ALONG_K | MM_BF16>;
    else if (am == MM_ALONG_K && bm == MM_BF16)
        kern = k_tc_mm<MM_ALONG_K, MM_BF16>;
    else if (am == 0 && bm == MM_BF16)
        kern = k_tc_mm<0, MM_BF16>;
    if (!kern || (b_ones >= 0 && (bm & MM_ALONG_K) != 0)) return cudaErrorNotSupported;
    const int np = (N + 15) / 16 * 16;
    const size_t smem = tc::mm_smem_bytes(np);
    // never lowered: the training step's launches are captured into a graph
    // with their own sizes
    cudaError_t e = raise_smem_limit(kern, smem);
    if (e != cudaSuccess) return e;
    const int64_t slices = (K + kc - 1) / kc;
    // the output: part (dense [slices][M][ldc] partials) whenever it is given,
    // which it must be for more than one slice; C otherwise
    if ((slices > 1 && !part) || (!part && !C)) return cudaErrorInvalidValue;
    const MmOp a{A, sam, sak, a_bf16, -1}, b{B, sbn, sbk, b_bf16, b_ones};
    const dim3 grid((unsigned)((M + MM_M - 1) / MM_M), 1, (unsigned)slices);
    note_launch();
    kern<<<grid, MM_THREADS, smem, st>>>(a, b, C, ldc, M, N, np, K, kc, part, status);
    return cudaGetLastError();
}

}  // namespace cc
