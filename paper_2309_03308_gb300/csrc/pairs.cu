// Pearson/Spearman and binned MI on batches of point pairs (Section 3.2), the seeded pair sampler
// (Section 3.1) and per-segment extremes (Section 3, brick-pair maximum).
#include "device.cuh"
#include "internal.cuh"

namespace cc {

constexpr int kWarpsPerBlock = 8;

static unsigned pair_grid(int64_t N, int warps_per_block) {
    const int sms = sm_count();
    int64_t want = (N + warps_per_block - 1) / warps_per_block;
    int64_t cap = (int64_t)sms * 16;
    return (unsigned)(want < cap ? (want < 1 ? 1 : want) : cap);
}

// ----------------------------------------------------------------------------
// Pearson / Spearman on a pair batch: r = sum_m zhat_a[m] * zhat_b[m] with
// zhat the unit-norm centred vector (PPMCC, Section 3.2); on the rank plane
// this is Spearman. One warp per pair; VEC = 4 reads each row as float4.
template <int VEC>
__global__ void __launch_bounds__(kWarpsPerBlock * 32)
    k_pearson_pairs(const float* __restrict__ A, int64_t Pa, const float* __restrict__ B,
                    int64_t Pb, int n_pad, const uint32_t* __restrict__ pa,
                    const uint32_t* __restrict__ pb, int64_t N, float* __restrict__ out,
                    int* status) {
    const int lane = threadIdx.x & 31;
    const int64_t w0 = (int64_t)blockIdx.x * kWarpsPerBlock + (threadIdx.x >> 5);
    const int64_t stride = (int64_t)gridDim.x * kWarpsPerBlock;
    for (int64_t t = w0; t < N; t += stride) {
        const uint32_t p = pa[t], q = pb[t];
        if (p >= Pa || q >= Pb) {
            if (lane == 0) {
                out[t] = CUDART_NAN_F;
                set_status(status, DEV_BAD_INDEX);
            }
            continue;
        }
        const float* a = A + (int64_t)p * n_pad;
        const float* b = B + (int64_t)q * n_pad;
        float acc = 0.f;
        if (VEC == 4) {
            for (int m = lane * 4; m < n_pad; m += 128) {
                const float4 u = __ldg(reinterpret_cast<const float4*>(a + m));
                const float4 v = __ldg(reinterpret_cast<const float4*>(b + m));
                acc = fmaf(u.x, v.x, acc);
                acc = fmaf(u.y, v.y, acc);
                acc = fmaf(u.z, v.z, acc);
                acc = fmaf(u.w, v.w, acc);
            }
        } else {
            for (int m = lane; m < n_pad; m += 32) acc = fmaf(__ldg(a + m), __ldg(b + m), acc);
        }
        acc = warp_sum_f32(acc);
        if (lane == 0) out[t] = acc;
    }
}

cudaError_t launch_pearson_pairs(const float* plane_a, int64_t Pa, const float* plane_b,
                                 int64_t Pb, int n_pad, const uint32_t* pa, const uint32_t* pb,
                                 int64_t N, float* out, int* status, cudaStream_t st) {
    if (N <= 0) return cudaSuccess;
    const unsigned g = pair_grid(N, kWarpsPerBlock);
    note_launch();
    if (n_pad % 128 == 0)
        k_pearson_pairs<4><<<g, kWarpsPerBlock * 32, 0, st>>>(plane_a, Pa, plane_b, Pb, n_pad, pa,
                                                             pb, N, out, status);
    else
        k_pearson_pairs<1><<<g, kWarpsPerBlock * 32, 0, st>>>(plane_a, Pa, plane_b, Pb, n_pad, pa,
                                                             pb, N, out, status);
    return cudaGetLastError();
}

// Joint-histogram sum of c ln c over the occupied cells for n > 128 members:
// up to 8 slices of 128 members, 4 per lane each; cells are recomputed from
// the (L1-resident) bin words when the owners read and clear them.
__device__ __forceinline__ long long hist_slices(const uint32_t* __restrict__ ba,
                                                 const uint32_t* __restrict__ bb, int n, int B,
                                                 int* h, const long long* clogc, int lane) {
    auto cell_of = [&](int c, int j) {
        const int w = (c * 128 >> 2) + lane;
        const uint32_t wa = __ldg(ba + w), wb = __ldg(bb + w);
        return (int)((wa >> (8 * j)) & 0xffu) * B + (int)((wb >> (8 * j)) & 0xffu);
    };
    unsigned own = 0;  // bit 4c + j: member 128c + 4 lane + j owns its cell
    for (int c = 0; c * 128 < n; ++c) {
        const int m = c * 128 + 4 * lane;
        if (m < n) {
#pragma unroll
            for (int j = 0; j < 4; ++j)
                if (m + j < n && atomicAdd(&h[cell_of(c, j)], 1) == 0) own |= 1u << (4 * c + j);
        }
    }
    __syncwarp();
    long long s = 0;
    for (unsigned o = own; o; o &= o - 1) {
        const int bit = __ffs(o) - 1;
        s += clogc[h[cell_of(bit >> 2, bit & 3)]];
    }
    __syncwarp();
    for (unsigned o = own; o; o &= o - 1) {
        const int bit = __ffs(o) - 1;
        h[cell_of(bit >> 2, bit & 3)] = 0;
    }
    __syncwarp();
    return s;
}

// ----------------------------------------------------------------------------
// Joint-histogram MI (Section 3.2, binning; Eq. 1 on the empirical
// distribution): with joint counts c_xy and marginals c_x, c_y,
//   MI = ln n + (1/n) [sum c_xy ln c_xy - sum c_x ln c_x - sum c_y ln c_y].
// The marginal sums are precomputed per point; c ln c comes from a
// fixed-point table so the sum is exact and order independent.
// One warp per pair; the B x B histogram lives in shared memory. Each lane
// reads four members' bins as one 32-bit word per side; the sample whose
// atomic increment found its cell empty owns the cell and, once the counts
// are complete, adds that cell's c ln c and clears it, so every occupied cell
// is summed once and no sweep over the B^2 cells is needed. A warp keeps the
// fixed-point sums of 32 consecutive pairs of its own, one per lane, and
// converts them to MI together: the FP64 steps (GB300's FP64 pipe is narrow)
// then run once per 32 pairs instead of once per pair on one lane.
__global__ void __launch_bounds__(kWarpsPerBlock * 32)
    k_hist_pairs(const uint8_t* __restrict__ bins_a, const long long* __restrict__ hm_a,
                 int64_t Pa, const uint8_t* __restrict__ bins_b,
                 const long long* __restrict__ hm_b, int64_t Pb, int n, int n_pad, int B,
                 const long long* __restrict__ clogc_fix, double logn, double fix_over_n,
                 const uint32_t* __restrict__ pa, const uint32_t* __restrict__ pb, int64_t N,
                 float* __restrict__ out, int* status) {
    __shared__ int hist[kWarpsPerBlock][256];
    extern __shared__ long long clogc[];  // [n + 1]
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    int* h = hist[warp];
    for (int c = threadIdx.x; c < 256 * kWarpsPerBlock; c += blockDim.x) (&hist[0][0])[c] = 0;
    for (int c = threadIdx.x; c <= n; c += blockDim.x) clogc[c] = clogc_fix[c];
    __syncthreads();
    const int64_t w0 = (int64_t)blockIdx.x * kWarpsPerBlock + warp;
    const int64_t stride = (int64_t)gridDim.x * kWarpsPerBlock;
    long long dk = 0;   // this lane's pending pair: fixed-point sum difference
    int64_t tk = -1;    // and its index
    int slot = 0;       // lane that takes the next pair
    auto flush = [&]() {
        if (tk >= 0) out[tk] = (float)(logn + (double)dk * fix_over_n);
        tk = -1;
        slot = 0;
    };
    for (int64_t t = w0; t < N; t += stride) {
        const uint32_t p = pa[t], q = pb[t];
        if (p >= Pa || q >= Pb) {
            if (lane == 0) {
                out[t] = CUDART_NAN_F;
                set_status(status, DEV_BAD_INDEX);
            }
            continue;
        }
        const uint32_t* ba = reinterpret_cast<const uint32_t*>(bins_a + (int64_t)p * n_pad);
        const uint32_t* bb = reinterpret_cast<const uint32_t*>(bins_b + (int64_t)q * n_pad);
        long long s = 0;
        if (n <= 128) {  // one slice: cells stay in registers
            const int m = 4 * lane;
            uint32_t wa = 0, wb = 0;
            if (m < n) {
                wa = __ldg(ba + lane);
                wb = __ldg(bb + lane);
            }
            int cell[4];
            unsigned own = 0;
#pragma unroll
            for (int j = 0; j < 4; ++j) {
                cell[j] = (int)((wa >> (8 * j)) & 0xffu) * B + (int)((wb >> (8 * j)) & 0xffu);
                if (m + j < n && atomicAdd(&h[cell[j]], 1) == 0) own |= 1u << j;
            }
            __syncwarp();
#pragma unroll
            for (int j = 0; j < 4; ++j)
                if ((own >> j) & 1u) s += clogc[h[cell[j]]];
            __syncwarp();
#pragma unroll
            for (int j = 0; j < 4; ++j)
                if ((own >> j) & 1u) h[cell[j]] = 0;
            __syncwarp();
        } else {
            s = hist_slices(ba, bb, n, B, h, clogc, lane);
        }
        s = warp_sum_u64_redux(s);  // c ln c >= 0: the fixed-point sums are non-negative
        if (lane == slot) {
            dk = s - hm_a[p] - hm_b[q];
            tk = t;
        }
        if (++slot == 32) flush();
    }
    flush();
}

cudaError_t launch_hist_pairs(const uint8_t* bins_a, const int64_t* hm_a, int64_t Pa,
                              const uint8_t* bins_b, const int64_t* hm_b, int64_t Pb, int n,
                              int n_pad, int B, const int64_t* clogc_fix, const uint32_t* pa,
                              const uint32_t* pb, int64_t N, float* out, int* status,
                              cudaStream_t st) {
    if (N <= 0) return cudaSuccess;
    const unsigned g = pair_grid(N, kWarpsPerBlock);
    note_launch();
    k_hist_pairs<<<g, kWarpsPerBlock * 32, (n + 1) * sizeof(long long), st>>>(
        bins_a, (const long long*)hm_a, Pa, bins_b, (const long long*)hm_b, Pb, n, n_pad, B,
        (const long long*)clogc_fix, std::log((double)n), 1.0 / (kFixScale * n), pa, pb, N, out,
        status);
    return cudaGetLastError();
}

// ----------------------------------------------------------------------------
// Uniform pair sampler (Section 3.1) on Philox4x64-10 (device.cuh).
__global__ void k_sample_pairs(const uint32_t* __restrict__ pts_a, int64_t na,
                               const uint32_t* __restrict__ pts_b, int64_t nb, int self,
                               uint64_t seed, uint64_t sstream, uint64_t first, int64_t N,
                               uint32_t* __restrict__ pa, uint32_t* __restrict__ pb) {
    for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < N;
         t += (int64_t)gridDim.x * blockDim.x) {
        uint64_t c[4] = {first + (uint64_t)t, 0, 0, 0};
        philox4x64_10(c, seed, sstream);
        uint64_t a = __umul64hi(c[0], (uint64_t)na), b;
        if (self) {
            b = __umul64hi(c[1], (uint64_t)na - 1);
            b += (b >= a);
            if (b < a) {
                const uint64_t tmp = a;
                a = b;
                b = tmp;
            }
        } else {
            b = __umul64hi(c[1], (uint64_t)nb);
        }
        pa[t] = pts_a[a];
        pb[t] = pts_b[b];
    }
}

// Quasi-random pair samplers (Section 3.1): Halton radical inverses in exact
// integer arithmetic, or the R6 Kronecker sequence in IEEE double; the exact
// mapping to voxels is stated with cc_sample_pairs_lds in the header.
struct LdsArgs {
    int kind, self;
    int ext[6];
    double alpha[6];
};

__global__ void k_sample_lds(LdsArgs g, const uint32_t* __restrict__ pts_a,
                             const uint32_t* __restrict__ pts_b, uint64_t first, int64_t N,
                             uint32_t* __restrict__ pa, uint32_t* __restrict__ pb) {
    const int bases[6] = {2, 3, 5, 7, 11, 13};
    for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < N;
         t += (int64_t)gridDim.x * blockDim.x) {
        const uint64_t j = first + (uint64_t)t + 1;
        int64_t c[6];
#pragma unroll
        for (int d = 0; d < 6; ++d) {
            if (g.kind == 1) {
                const uint64_t b = (uint64_t)bases[d];
                uint64_t jj = j, num = 0, den = 1;
                while (jj > 0) {
                    num = num * b + jj % b;
                    jj /= b;
                    den *= b;
                }
                c[d] = (int64_t)((num * (uint64_t)g.ext[d]) / den);
            } else {
                double u = __dadd_rn(0.5, __dmul_rn((double)j, g.alpha[d]));
                u = u - floor(u);
                const int64_t v = (int64_t)floor(__dmul_rn(u, (double)g.ext[d]));
                c[d] = v < g.ext[d] - 1 ? v : g.ext[d] - 1;
            }
        }
        const int64_t na = (int64_t)g.ext[0] * g.ext[1] * g.ext[2];
        int64_t a = c[0] + g.ext[0] * (c[1] + g.ext[1] * c[2]);
        int64_t b = c[3] + g.ext[3] * (c[4] + g.ext[4] * c[5]);
        if (g.self) {
            if (a == b) b = (b + 1) % na;
            if (b < a) {
                const int64_t tmp = a;
                a = b;
                b = tmp;
            }
        }
        pa[t] = pts_a[a];
        pb[t] = pts_b[b];
    }
}

cudaError_t launch_sample_lds(int kind, const int* ext, const double* alpha, int self,
                              const uint32_t* pts_a, const uint32_t* pts_b, uint64_t first,
                              int64_t N, uint32_t* pa, uint32_t* pb, cudaStream_t st) {
    if (N <= 0) return cudaSuccess;
    LdsArgs g;
    g.kind = kind;
    g.self = self;
    for (int d = 0; d < 6; ++d) {
        g.ext[d] = ext[d];
        g.alpha[d] = alpha[d];
    }
    int64_t blocks = (N + 255) / 256;
    const int64_t cap = (int64_t)sm_count() * 32;
    if (blocks > cap) blocks = cap;
    note_launch();
    k_sample_lds<<<(unsigned)blocks, 256, 0, st>>>(g, pts_a, pts_b, first, N, pa, pb);
    return cudaGetLastError();
}

cudaError_t launch_sample_pairs(const uint32_t* pts_a, int64_t na, const uint32_t* pts_b,
                                int64_t nb, int self, uint64_t seed, uint64_t stream,
                                uint64_t first, int64_t N, uint32_t* pa, uint32_t* pb,
                                cudaStream_t st) {
    if (N <= 0) return cudaSuccess;
    int64_t blocks = (N + 255) / 256;
    const int64_t cap = (int64_t)sm_count() * 32;
    if (blocks > cap) blocks = cap;
    note_launch();
    k_sample_pairs<<<(unsigned)blocks, 256, 0, st>>>(pts_a, na, pts_b, nb, self, seed, stream,
                                                     first, N, pa, pb);
    return cudaGetLastError();
}

// ----------------------------------------------------------------------------
// Extremes per segment of a value batch (Section 3: brick-pair maximum over
// its evaluated point pairs; minimum too, Section 5.3). Two levels: one CTA
// per chunk of at most kChunk values, then one warp per segment folds its
// chunks. Ties resolve to the smallest batch index.
__global__ void __launch_bounds__(256)
    k_chunk_extremes(const float* __restrict__ v, const int64_t* __restrict__ bounds,
                     Partial* __restrict__ part) {
    __shared__ Ext red[8];
    const int64_t lo = bounds[2 * blockIdx.x], hi = bounds[2 * blockIdx.x + 1];
    Ext e = ext_empty();
    for (int64_t t = lo + threadIdx.x; t < hi; t += blockDim.x) ext_add(e, v[t], (unsigned long long)t);
    e = warp_ext(e);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = e;
    __syncthreads();
    if (threadIdx.x == 0) {
        Ext r = red[0];
        for (int w = 1; w < 8; ++w)
            ext_merge(r, red[w].vmax, red[w].imax, red[w].vmin, red[w].imin, red[w].count);
        part[blockIdx.x] = Partial{r.vmax, r.vmin, r.imax, r.imin, r.count};
    }
}

__global__ void k_fold_segments(const Partial* __restrict__ part, const int64_t* __restrict__ first,
                                int n_seg, Partial* __restrict__ out) {
    const int lane = threadIdx.x & 31;
    const int s = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
    if (s >= n_seg) return;
    Ext e = ext_empty();
    for (int64_t c = first[s] + lane; c < first[s + 1]; c += 32)
        ext_merge(e, part[c].max, part[c].argmax, part[c].min, part[c].argmin, part[c].count);
    e = warp_ext(e);
    if (lane == 0) out[s] = Partial{e.vmax, e.vmin, e.imax, e.imin, e.count};
}

cudaError_t launch_segment_extremes(const float* values, const int64_t* chunk_bounds,
                                    int64_t n_chunks, const int64_t* seg_first_chunk, int n_seg,
                                    Partial* chunk_part, Partial* out, cudaStream_t st) {
    if (n_chunks > 0) {
        note_launch();
        k_chunk_extremes<<<(unsigned)n_chunks, 256, 0, st>>>(values, chunk_bounds, chunk_part);
        cudaError_t e = cudaGetLastError();
        if (e != cudaSuccess) return e;
    }
    if (n_seg <= 0) return cudaSuccess;
    note_launch();
    k_fold_segments<<<(n_seg + 7) / 8, 256, 0, st>>>(chunk_part, seg_first_chunk, n_seg, out);
    return cudaGetLastError();
}

}  // namespace cc
