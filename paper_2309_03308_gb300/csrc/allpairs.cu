// All pairs between two regions in FP32 on the SIMT pipes (Section 4.2: the
// focus view's exhaustive refinement of one brick pair; Section 3: the brick
// pair's indicator is the maximum over its point pairs).
//
// R = Z_A^T Z_B with Z the member-major unit-norm centred planes [nk][np_pad]
// of the two regions: every output is a PPMCC (or Spearman on rank planes).
// The epilogue optionally stores every value and always reduces the tile to
// (max, argmax, min, argmin, count); a second kernel folds the per-tile
// partials. Pairs of a self region pair reduce only a < b.
//
// Tiling: 128 x 128 outputs per CTA, 256 threads with 8 x 8 outputs each
// (rows ty*4+{0..3} and 64+ty*4+{0..3}, same for columns), K staged through a
// 3-deep cp.async ring of 8-member slices. The products accumulate with the
// packed FP32 FMA (two IEEE fp32 fma.rn per instruction on adjacent columns),
// which halves the issue slots the FMAs take; the values are those of plain
// fmaf in the same order.
#include "device.cuh"
#include "internal.cuh"

namespace cc {

constexpr int BM = 128, BN = 128, KC = 8, STAGES = 3, NT = 256;

__device__ __forceinline__ void cp_async16(void* smem, const void* gmem) {
    const unsigned s = (unsigned)__cvta_generic_to_shared(smem);
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(s), "l"(gmem));
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::); }
template <int N>
__device__ __forceinline__ void cp_async_wait() {
    asm volatile("cp.async.wait_group %0;\n" ::"n"(N));
}

__global__ void __launch_bounds__(NT, 2)
    k_allpairs_f32(const float* __restrict__ A, int64_t lda, const float* __restrict__ B,
                   int64_t ldb, int nk, int64_t PA, int64_t PB, int self, float* __restrict__ C,
                   int64_t ldc, int vec_store, Partial* __restrict__ partials) {
    __shared__ __align__(16) float As[STAGES][KC][BM];
    __shared__ __align__(16) float Bs[STAGES][KC][BN];
    __shared__ Ext red[NT / 32];

    const int tid = threadIdx.x;
    const int tx = tid & 15, ty = tid >> 4;
    const int64_t a0 = (int64_t)blockIdx.y * BM, b0 = (int64_t)blockIdx.x * BN;
    const int64_t tile_id = (int64_t)blockIdx.y * gridDim.x + blockIdx.x;

    if (self && !C && b0 + BN - 1 <= a0) {  // nothing to store and no pair a < b here
        if (tid == 0) {
            Partial e;
            e.max = -CUDART_INF_F;
            e.min = CUDART_INF_F;
            e.argmax = e.argmin = ~0ull;
            e.count = 0;
            partials[tile_id] = e;
        }
        return;
    }

    const int lrow = tid >> 5, lcol = (tid & 31) * 4;
    const int nkt = nk / KC;
    auto load_stage = [&](int s, int kt) {
        const int k = kt * KC + lrow;
        cp_async16(&As[s][lrow][lcol], A + (int64_t)k * lda + a0 + lcol);
        cp_async16(&Bs[s][lrow][lcol], B + (int64_t)k * ldb + b0 + lcol);
    };

    // accumulators in column pairs for the packed FP32 FMA (fma.rn.f32x2:
    // two independent IEEE fp32 FMAs per instruction)
    unsigned long long acc2[8][4];
#pragma unroll
    for (int i = 0; i < 8; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) acc2[i][j] = 0ull;

#pragma unroll
    for (int s = 0; s < STAGES - 1; ++s) {
        if (s < nkt) load_stage(s, s);
        cp_async_commit();
    }
    for (int kt = 0; kt < nkt; ++kt) {
        cp_async_wait<STAGES - 2>();
        __syncthreads();
        const int nxt = kt + STAGES - 1;
        if (nxt < nkt) load_stage(nxt % STAGES, nxt);
        cp_async_commit();
        const int s = kt % STAGES;
#pragma unroll
        for (int kk = 0; kk < KC; ++kk) {
            const float4 al = *reinterpret_cast<const float4*>(&As[s][kk][ty * 4]);
            const float4 ah = *reinterpret_cast<const float4*>(&As[s][kk][64 + ty * 4]);
            const float4 bl = *reinterpret_cast<const float4*>(&Bs[s][kk][tx * 4]);
            const float4 bh = *reinterpret_cast<const float4*>(&Bs[s][kk][64 + tx * 4]);
            const float a[8] = {al.x, al.y, al.z, al.w, ah.x, ah.y, ah.z, ah.w};
            const unsigned long long bp[4] = {pack2(bl.x, bl.y), pack2(bl.z, bl.w),
                                              pack2(bh.x, bh.y), pack2(bh.z, bh.w)};
#pragma unroll
            for (int i = 0; i < 8; ++i) {
                const unsigned long long aa = pack2(a[i], a[i]);
#pragma unroll
                for (int j = 0; j < 4; ++j) ffma2(acc2[i][j], aa, bp[j]);
            }
        }
    }
    cp_async_wait<0>();
    float acc[8][8];
#pragma unroll
    for (int i = 0; i < 8; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) unpack2(acc2[i][j], acc[i][2 * j], acc[i][2 * j + 1]);

    // epilogue: store and reduce. A tile inside both regions and clear of the
    // self-pair diagonal reduces without per-value checks: value extremes
    // with the thread-local position (compile-time), first position on ties,
    // which is the smallest linear pair index (rows, then columns, ascend).
    Ext e = ext_empty();
    const bool interior = a0 + BM <= PA && b0 + BN <= PB && (!self || b0 >= a0 + BM);
    if (interior) {
        float vmax = -CUDART_INF_F, vmin = CUDART_INF_F;
        int pmax = 0, pmin = 0;
#pragma unroll
        for (int i = 0; i < 8; ++i) {
#pragma unroll
            for (int hj = 0; hj < 8; ++hj) {
                const float v = acc[i][hj];
                pmax = v > vmax ? i * 8 + hj : pmax;
                vmax = fmaxf(vmax, v);
                pmin = v < vmin ? i * 8 + hj : pmin;
                vmin = fminf(vmin, v);
            }
        }
        auto lin = [&](int pos) {
            const int i = pos >> 3, hj = pos & 7;
            const int64_t row = a0 + (i < 4 ? ty * 4 + i : 64 + ty * 4 + (i - 4));
            const int64_t col = b0 + (hj >> 2) * 64 + tx * 4 + (hj & 3);
            return (unsigned long long)(row * PB + col);
        };
        e.vmax = vmax;
        e.vmin = vmin;
        e.imax = lin(pmax);
        e.imin = lin(pmin);
        e.count = 64;
    }
#pragma unroll
    for (int i = 0; i < 8; ++i) {
        const int64_t row = a0 + (i < 4 ? ty * 4 + i : 64 + ty * 4 + (i - 4));
        if (row >= PA) continue;
#pragma unroll
        for (int h = 0; h < 2; ++h) {
            const int64_t col0 = b0 + h * 64 + tx * 4;
            if (C) {
                float* dst = C + row * ldc + col0;
                if (vec_store && col0 + 3 < PB) {
                    __stcs(reinterpret_cast<float4*>(dst),
                           make_float4(acc[i][h * 4], acc[i][h * 4 + 1], acc[i][h * 4 + 2],
                                       acc[i][h * 4 + 3]));
                } else {
#pragma unroll
                    for (int j = 0; j < 4; ++j)
                        if (col0 + j < PB) __stcs(dst + j, acc[i][h * 4 + j]);
                }
            }
            if (!interior) {
#pragma unroll
                for (int j = 0; j < 4; ++j) {
                    const int64_t col = col0 + j;
                    if (col < PB && (!self || row < col))
                        ext_add(e, acc[i][h * 4 + j], (unsigned long long)(row * PB + col));
                }
            }
        }
    }
    e = warp_ext(e);
    if ((tid & 31) == 0) red[tid >> 5] = e;
    __syncthreads();
    if (tid == 0) {
        Ext t = red[0];
        for (int w = 1; w < NT / 32; ++w)
            ext_merge(t, red[w].vmax, red[w].imax, red[w].vmin, red[w].imin, red[w].count);
        Partial out;
        out.max = t.vmax;
        out.min = t.vmin;
        out.argmax = t.imax;
        out.argmin = t.imin;
        out.count = t.count;
        partials[tile_id] = out;
    }
}

// Fold per-tile partials into one result (one CTA).
__global__ void k_fold_partials(const Partial* __restrict__ p, int64_t n, Partial* __restrict__ r) {
    __shared__ Ext red[32];
    Ext e = ext_empty();
    for (int64_t i = threadIdx.x; i < n; i += blockDim.x)
        ext_merge(e, p[i].max, p[i].argmax, p[i].min, p[i].argmin, p[i].count);
    e = warp_ext(e);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = e;
    __syncthreads();
    if (threadIdx.x == 0) {
        Ext t = red[0];
        for (int w = 1; w < (int)(blockDim.x >> 5); ++w)
            ext_merge(t, red[w].vmax, red[w].imax, red[w].vmin, red[w].imin, red[w].count);
        r->max = t.vmax;
        r->min = t.vmin;
        r->argmax = t.imax;
        r->argmin = t.imin;
        r->count = t.count;
    }
}

size_t allpairs_partials(int64_t PA, int64_t PB) {
    return (size_t)((PA + BM - 1) / BM) * (size_t)((PB + BN - 1) / BN);
}

cudaError_t launch_allpairs_f32(const float* A, int64_t lda, const float* B, int64_t ldb, int nk,
                                int64_t PA, int64_t PB, int self, float* C, int64_t ldc,
                                Partial* partials, Partial* result, cudaStream_t st) {
    const int64_t ta = (PA + BM - 1) / BM, tb = (PB + BN - 1) / BN;
    const int vec_store = C && (ldc % 4 == 0) && (((uintptr_t)C & 15) == 0);
    dim3 grid((unsigned)tb, (unsigned)ta);
    note_launch();
    k_allpairs_f32<<<grid, NT, 0, st>>>(A, lda, B, ldb, nk, PA, PB, self, C, ldc, vec_store,
                                        partials);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    note_launch();
    k_fold_partials<<<1, 1024, 0, st>>>(partials, ta * tb, result);
    return cudaGetLastError();
}

}  // namespace cc

// ----------------------------------------------------------------------------
// Allocation-free variant of the all-pairs extremes (cc_all_pairs_static).
// The per-tile partials live in a file-scope device array instead of context
// scratch; the caller passes the standardized planes and the output.
#include <mutex>

namespace {

constexpr int64_t kStaticTiles = 1 << 16;  // 65,536 tiles of 128 x 128 pairs (2.5 MiB)
__device__ __align__(256) cc::Partial g_static_partials[kStaticTiles];

std::mutex g_static_mu;
constexpr int kMaxDevices = 64;
cc::Partial* g_static_addr[kMaxDevices] = {};

static_assert(sizeof(cc::Partial) == sizeof(cc_rp_result), "result layout");
static_assert(offsetof(cc::Partial, argmax) == offsetof(cc_rp_result, argmax), "result layout");
static_assert(offsetof(cc::Partial, count) == offsetof(cc_rp_result, count), "result layout");

// Device address of the static partials on the current device; resolved
// once per device with that device current.
cudaError_t static_partials(cc::Partial** out) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
    std::lock_guard<std::mutex> lock(g_static_mu);
    if (!g_static_addr[dev]) {
        void* p = nullptr;
        e = cudaGetSymbolAddress(&p, g_static_partials);
        if (e != cudaSuccess) return e;
        g_static_addr[dev] = static_cast<cc::Partial*>(p);
    }
    *out = g_static_addr[dev];
    return cudaSuccess;
}

}  // namespace

extern "C" cc_status cc_all_pairs_static(const float* za, int64_t lda, const float* zb, int64_t ldb,
                                         int nk, int64_t na, int64_t nb, int self, float* values,
                                         int64_t ldv, cc_rp_result* out, void* stream) {
    if (!za || !zb || !out || nk < 8 || nk % 8 != 0 || na < 1 || nb < 1)
        return CC_ERR_INVALID_ARG;
    const int64_t ta = (na + cc::BM - 1) / cc::BM, tb = (nb + cc::BN - 1) / cc::BN;
    if (lda < ta * cc::BM || ldb < tb * cc::BN || lda % 4 || ldb % 4 ||
        ((uintptr_t)za & 15) || ((uintptr_t)zb & 15))
        return CC_ERR_INVALID_ARG;
    if (self && (za != zb || na != nb || lda != ldb)) return CC_ERR_INVALID_ARG;
    if (values && ldv < nb) return CC_ERR_INVALID_ARG;
    // beyond the static scratch (each factor is bounded before the product is formed)
    if (ta > 65535 || tb > kStaticTiles || ta * tb > kStaticTiles) return CC_ERR_INVALID_ARG;
    cc::Partial* parts = nullptr;
    cudaError_t e = static_partials(&parts);
    if (e == cudaSuccess)
        e = cc::launch_allpairs_f32(za, lda, zb, ldb, nk, na, nb, self, values, ldv, parts,
                                    reinterpret_cast<cc::Partial*>(out), (cudaStream_t)stream);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return CC_ERR_CUDA;
    }
    return CC_OK;
}
