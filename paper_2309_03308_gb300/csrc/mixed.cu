// Reduced-precision all-pairs with exact, certified extremes (project
// addition to the Section 4.2 focus refinement; Section 3: the brick pair's
// maximum).
//
//  1. quantize   each region point's unit-norm standardized vector to BF16, or
//                to FP8 E4M3 with scale 448 / max|z|; record the point's
//                quantization error norm e_p = || dequant(q_p) - z_p ||_2.
//  2. contract   on the tensor cores (tc_gemm.cu) -> per (row, 32-column chunk)
//                max / min of the approximate values r~.
//  3. select     the top chunks by chunk max (two 12-bit histogram passes on
//                order-preserving keys) and re-evaluate every pair in them with
//                Dot2 (Ogita, Rump, Oishi 2005: TwoProduct by FMA + TwoSum),
//                an almost exact fp32 dot product of the fp32 planes.
//  4. certify    |r~ - r| <= B for every pair, with B = 2 e + e^2 +
//                (1 + e)^2 2^-12 + 2^-20, e = max_p e_p (Cauchy-Schwarz on the
//                quantization errors plus a conservative accumulation term).
//                Any pair whose chunk max is below r* - B (r* = best refined
//                value) cannot beat r*; every chunk at or above it is refined
//                in a second pass, after which r* is the exact maximum.
//  5. top-K      of the refined values, sorted descending.
// The minimum runs the same passes on negated values.
#include <cuda_bf16.h>
#include <cuda_fp8.h>

#include "device.cuh"
#include "internal.cuh"

namespace cc {

__device__ __forceinline__ unsigned okey(float v) {
    const unsigned b = __float_as_uint(v + 0.0f);
    return (b & 0x80000000u) ? ~b : (b | 0x80000000u);
}
__device__ __forceinline__ float okey_inv(unsigned o) {
    return __uint_as_float((o & 0x80000000u) ? (o & 0x7fffffffu) : ~o);
}

// ---------------------------------------------------------------------------
// 1. quantization: one warp per region point. The error norms' maximum goes
// to emax_bits with one atomic per block (8 warps), not per warp: 20,480
// atomics on one address serialised and took most of the launch.
template <bool FP8>
__global__ void __launch_bounds__(256)
    k_quantize(const float* __restrict__ plane, int n_pad, int n, const uint32_t* __restrict__ pts,
               int64_t np, int64_t np_pad, int kbytes, unsigned char* __restrict__ q,
               float* __restrict__ inv_scale, unsigned* __restrict__ emax_bits) {
    __shared__ unsigned block_max[8];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int64_t r = (int64_t)blockIdx.x * 8 + warp;
    const int kelems = FP8 ? kbytes : kbytes / 2;
    unsigned char* qrow = q + r * kbytes;
    unsigned my_max = 0u;  // bits of this warp's error norm (non-negative floats order as bits)
    if (r < np_pad && r >= np) {  // warp-uniform: a padding row
        for (int b = lane * 4; b < kbytes; b += 128) *reinterpret_cast<uint32_t*>(qrow + b) = 0;
        if (FP8 && lane == 0) inv_scale[r] = 0.f;
    } else if (r < np) {  // warp-uniform
        const float* z = plane + (int64_t)pts[r] * n_pad;
        float amax = 0.f;
        if (FP8) {
            for (int k = lane; k < n; k += 32) amax = fmaxf(amax, fabsf(z[k]));
#pragma unroll
            for (int o = 16; o > 0; o >>= 1)
                amax = fmaxf(amax, __shfl_xor_sync(0xffffffffu, amax, o));
        }
        const float s = FP8 ? (amax > 0.f ? 448.f / amax : 1.f) : 1.f;
        float err = 0.f;
        for (int k = lane * 2; k < kelems; k += 64) {
            const float z0 = k < n ? z[k] : 0.f, z1 = k + 1 < n ? z[k + 1] : 0.f;
            float d0, d1;
            if (FP8) {
                const __nv_fp8x2_storage_t v = __nv_cvt_float2_to_fp8x2(
                    make_float2(z0 * s, z1 * s), __NV_SATFINITE, __NV_E4M3);
                *reinterpret_cast<__nv_fp8x2_storage_t*>(qrow + k) = v;
                const __half2_raw hr = __nv_cvt_fp8x2_to_halfraw2(v, __NV_E4M3);
                const float2 back = __half22float2(*reinterpret_cast<const __half2*>(&hr));
                d0 = back.x / s - z0;
                d1 = back.y / s - z1;
            } else {
                const __nv_bfloat162 v = __floats2bfloat162_rn(z0, z1);
                *reinterpret_cast<__nv_bfloat162*>(qrow + 2 * k) = v;
                const float2 back = __bfloat1622float2(v);
                d0 = back.x - z0;
                d1 = back.y - z1;
            }
            err = fmaf(d0, d0, fmaf(d1, d1, err));
        }
        err = warp_sum_f32(err);
        if (FP8 && lane == 0) inv_scale[r] = 1.f / s;
        // small relative margin for the fp32 accumulation of the error norm
        my_max = __float_as_uint(sqrtf(err) * 1.001f);
    }
    if (lane == 0) block_max[warp] = my_max;
    __syncthreads();
    if (threadIdx.x == 0) {
        unsigned m = 0u;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) m = max(m, block_max[w]);
        if (m) atomicMax(emax_bits, m);
    }
}

// 1b. Spearman, n <= 257: the centred doubled ranks c = rank2 - (n + 1) are
// integers with |c| <= n - 1 <= 256, exact in BF16, and every partial sum of
// their products is an integer below 2^24 (sum |c_a c_b| <= sum c^2 <= n^3 / 3),
// exact in FP32. The operand is c itself with the per-point scale
// 1 / sqrt(sum c^2) applied in the epilogue, so the contraction has no
// quantization error (e_p = 0).
__global__ void __launch_bounds__(256)
    k_quantize_ranks(const int16_t* __restrict__ rank2, int n_pad, int n,
                     const uint32_t* __restrict__ pts, int64_t np, int64_t np_pad, int kbytes,
                     unsigned char* __restrict__ q, float* __restrict__ inv_scale) {
    const int lane = threadIdx.x & 31;
    const int64_t r = (int64_t)blockIdx.x * 8 + (threadIdx.x >> 5);
    if (r >= np_pad) return;
    unsigned char* qrow = q + r * kbytes;
    if (r >= np) {
        for (int b = lane * 4; b < kbytes; b += 128) *reinterpret_cast<uint32_t*>(qrow + b) = 0;
        if (lane == 0) inv_scale[r] = 0.f;
        return;
    }
    const int16_t* c2 = rank2 + (int64_t)pts[r] * n_pad;
    long long ss = 0;
    for (int k = lane * 2; k < kbytes / 2; k += 64) {
        const int c0 = k < n ? c2[k] - (n + 1) : 0, c1 = k + 1 < n ? c2[k + 1] - (n + 1) : 0;
        *reinterpret_cast<__nv_bfloat162*>(qrow + 2 * k) =
            __floats2bfloat162_rn((float)c0, (float)c1);
        ss += (long long)(c0 * c0 + c1 * c1);
    }
    ss = warp_sum_i64(ss);
    if (lane == 0) inv_scale[r] = ss > 0 ? (float)rsqrt((double)ss) : 0.f;
}

// ---------------------------------------------------------------------------
// 3a. two-pass histogram select on order-preserving keys of sign * value,
// for NS = 1 or 2 value arrays at once (the maximum and the minimum side of a
// region pair share every pass). Pass `level` 0 bins the top 32 - shift bits
// (shift 20: 12 bits; 21: 11 bits, the histogram the tensor-core kernel
// builds), pass 1 the next 12 among keys whose top bits equal sel->prefix.
// Values of -inf (empty chunks) are skipped. N is a multiple of 4 (read as
// float4).
struct SideVals {
    const float* v[2];
    float sign[2];
    Select* sel[2];
    const float* lo_val[2];  // second compaction: the side's value threshold (else null)
};

template <int NS>
__global__ void __launch_bounds__(256)
    k_hist12(SideVals sv, int64_t N, int level, int shift, unsigned* __restrict__ hist,
             const unsigned* __restrict__ nchunks) {
    __shared__ unsigned h[NS][4096];
    if (nchunks) N = min(N, (int64_t)*nchunks * 32);
    for (int i = threadIdx.x; i < NS * 4096; i += blockDim.x) (&h[0][0])[i] = 0;
    __syncthreads();
    unsigned prefix[NS];
#pragma unroll
    for (int s = 0; s < NS; ++s) prefix[s] = level ? sv.sel[s]->prefix : 0u;
    const int64_t N4 = N / 4;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < N4;
         i += (int64_t)gridDim.x * blockDim.x) {
#pragma unroll
        for (int s = 0; s < NS; ++s) {
            const float4 q = reinterpret_cast<const float4*>(sv.v[s])[i];
            const float w[4] = {q.x, q.y, q.z, q.w};
#pragma unroll
            for (int j = 0; j < 4; ++j) {
                const float x = sv.sign[s] * w[j];
                if (!(x > -CUDART_INF_F)) continue;
                const unsigned k = okey(x);
                if (level == 0) atomicAdd(&h[s][k >> shift], 1u);
                else if ((k >> shift) == prefix[s]) atomicAdd(&h[s][(k >> (shift - 12)) & 0xfffu], 1u);
            }
        }
    }
    // the last N % 4 values
    for (int64_t i = 4 * N4 + (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < N;
         i += (int64_t)gridDim.x * blockDim.x) {
#pragma unroll
        for (int s = 0; s < NS; ++s) {
            const float x = sv.sign[s] * sv.v[s][i];
            if (!(x > -CUDART_INF_F)) continue;
            const unsigned k = okey(x);
            if (level == 0) atomicAdd(&h[s][k >> shift], 1u);
            else if ((k >> shift) == prefix[s]) atomicAdd(&h[s][(k >> (shift - 12)) & 0xfffu], 1u);
        }
    }
    __syncthreads();
    for (int i = threadIdx.x; i < NS * 4096; i += blockDim.x)
        if ((&h[0][0])[i]) atomicAdd(&hist[i], (&h[0][0])[i]);
}

// One block per side: scan the side's 4096 bins from the top until `want`
// keys are covered.
__global__ void k_pick_bin(unsigned* __restrict__ hist_all, int level, int shift, unsigned want0,
                           unsigned want1, SideVals sv) {
    __shared__ unsigned part[1024];
    unsigned* hist = hist_all + 4096 * blockIdx.x;
    Select* sel = sv.sel[blockIdx.x];
    const unsigned want = blockIdx.x ? want1 : want0;
    // bins are scanned in descending order: thread t owns bins 4095-4t .. 4092-4t
    const int t = threadIdx.x;
    unsigned s = 0;
    for (int j = 0; j < 4; ++j) s += hist[4095 - 4 * t - j];
    part[t] = s;
    __syncthreads();
    for (int o = 1; o < 1024; o <<= 1) {  // inclusive prefix sum
        const unsigned x = t >= o ? part[t - o] : 0u;
        __syncthreads();
        part[t] += x;
        __syncthreads();
    }
    const unsigned target = level == 0 ? want : sel->need;
    const unsigned before = t ? part[t - 1] : 0u;
    const bool last_group = t == 1023;
    if ((before < target && part[t] >= target) || (last_group && part[t] < target)) {
        unsigned acc = before;
        int bin = 4095 - 4 * t - 3;
        for (int j = 0; j < 4; ++j) {
            const int b = 4095 - 4 * t - j;
            if (acc + hist[b] >= target) {
                bin = b;
                break;
            }
            acc += hist[b];
        }
        if (level == 0) {
            sel->prefix = (unsigned)bin;
            sel->need = target - acc;
        } else {
            sel->threshold = (sel->prefix << shift) | ((unsigned)bin << (shift - 12));
        }
        if (part[t] < target) sel->threshold = 0u;  // fewer keys than wanted: take all
    }
    __syncthreads();
    for (int i = t; i < 4096; i += 1024) hist[i] = 0;  // ready for the next pass
}

// 3b. compact chunk ids whose key lies in [lo_key, hi_key) (hi_key 0 = no cap)
// into out + s * cap for every side s. First pass (lo_val null): keys >=
// sel->threshold. Second pass: keys in [okey(*lo_val), sel->threshold),
// appended after the first pass's; skipped for a side whose first pass took
// every key (threshold 0) or overflowed.
template <int NS>
__global__ void __launch_bounds__(256)
    k_compact(SideVals sv, int64_t N, uint32_t* __restrict__ out, unsigned cap,
              const unsigned* __restrict__ nchunks) {
    if (nchunks) N = min(N, (int64_t)*nchunks * 32);
    unsigned lo[NS], hi[NS];
    bool on[NS];
    bool any = false;
#pragma unroll
    for (int s = 0; s < NS; ++s) {
        const Select* sel = sv.sel[s];
        const float* thr = sv.lo_val[s];
        on[s] = !(thr && (sel->threshold == 0u || sel->overflow));
        lo[s] = thr ? okey(*thr) : sel->threshold;
        hi[s] = thr ? sel->threshold : 0u;
        // second pass: an empty window [lo, hi) takes nothing (the usual case:
        // the first pass's threshold lies below the best value minus the bound)
        if (thr && lo[s] >= hi[s]) on[s] = false;
        any = any || on[s];
    }
    if (!any) return;  // the same for every thread
    const int lane = threadIdx.x & 31;
    auto offer = [&](int s, float w, int64_t idx) {
        const float x = sv.sign[s] * w;
        const unsigned k = okey(x);
        if (x > -CUDART_INF_F && k >= lo[s] && (hi[s] == 0u || k < hi[s])) {
            // one counter update per warp: the leader takes the warp's slots
            const unsigned m = __activemask();
            const int leader = __ffs(m) - 1;
            unsigned base = 0;
            if (lane == leader) base = atomicAdd(&sv.sel[s]->count, (unsigned)__popc(m));
            base = __shfl_sync(m, base, leader);
            const unsigned slot = base + __popc(m & ((1u << lane) - 1u));
            if (slot < cap) out[(size_t)s * cap + slot] = (uint32_t)idx;
            else atomicAdd(&sv.sel[s]->overflow, 1u);
        }
    };
    const int64_t N4 = N / 4;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < N4;
         i += (int64_t)gridDim.x * blockDim.x) {
#pragma unroll
        for (int s = 0; s < NS; ++s) {
            if (!on[s]) continue;
            const float4 q = reinterpret_cast<const float4*>(sv.v[s])[i];
            offer(s, q.x, 4 * i);
            offer(s, q.y, 4 * i + 1);
            offer(s, q.z, 4 * i + 2);
            offer(s, q.w, 4 * i + 3);
        }
    }
    for (int64_t i = 4 * N4 + (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < N;
         i += (int64_t)gridDim.x * blockDim.x) {
#pragma unroll
        for (int s = 0; s < NS; ++s)
            if (on[s]) offer(s, sv.v[s][i], i);
    }
}

// ---------------------------------------------------------------------------
// 3c. Dot2 re-evaluation of every pair in the candidate chunks. Chunk id i
// addresses cm[chunk][row] = i, i.e. chunk = i / na_pad, row = i % na_pad.
// One warp per chunk: the warp holds row a's member vector (n <= 1024) in
// registers and evaluates its 32 pairs (a, 32 * chunk + j).
// R = member slices of 32 in use (ceil(n / 32) rounded up to a power of two),
// a template parameter so every load of a row is issued before the sums.
template <int R>
__device__ __forceinline__ float dot2_warp(const float (&x)[R], const float* __restrict__ y,
                                           int n) {
    const int lane = threadIdx.x & 31;
    float s = 0.f, c = 0.f;
#pragma unroll
    for (int r = 0; r < R; ++r) {
        const int k = r * 32 + lane;
        if (k < n) {
            const float p = __fmul_rn(x[r], y[k]);
            const float pe = fmaf(x[r], y[k], -p);  // TwoProduct error, exact
            float t, q;
            two_sum(s, p, t, q);
            s = t;
            c = __fadd_rn(c, __fadd_rn(q, pe));
        }
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        const float s2 = __shfl_xor_sync(0xffffffffu, s, o);
        const float c2 = __shfl_xor_sync(0xffffffffu, c, o);
        float t, q;
        two_sum(s, s2, t, q);
        s = t;
        c = __fadd_rn(__fadd_rn(c, c2), q);
    }
    return __fadd_rn(s, c);
}

// One warp per chunk, one lane per pair: lane j evaluates (a, 32 * chunk + j)
// with a sequential Dot2 over the members. Lane j reads its own column row
// as aligned float4s (rows are n_pad >= 32 R floats, 16-byte aligned), two
// 32-member slices in flight at a time, and row a's member is broadcast from
// the lane that holds it, so a chunk costs two memory round trips, no shared
// memory and no reductions.
// The chunks of one side (blockIdx.y) of the refinement: candidate ids,
// where this pass's ids start (null: 0) and end, the sign of the side, and
// where the refined values, pair ids and the best key go.
struct RefineSide {
    const uint32_t* ids;
    const unsigned* start;
    const unsigned* count;
    float sign;
    float* vals;
    unsigned long long* pair_ids;
    unsigned long long* best;
};
struct RefineArgs {
    RefineSide s[2];
};

template <int R>
__global__ void __launch_bounds__(256)
    k_refine_chunks(const float* __restrict__ plane_a, const float* __restrict__ plane_b,
                    int n_pad, int n, const uint32_t* __restrict__ pts_a, int64_t na,
                    const uint32_t* __restrict__ pts_b, int64_t nb, int self, int64_t na_pad,
                    unsigned cap, RefineArgs args) {
    const RefineSide& rs = args.s[blockIdx.y];
    const uint32_t* __restrict__ ids = rs.ids;
    const unsigned* __restrict__ start_p = rs.start;
    const unsigned* __restrict__ count_p = rs.count;
    const float sign = rs.sign;
    float* __restrict__ vals = rs.vals;
    unsigned long long* __restrict__ pair_ids = rs.pair_ids;
    unsigned long long* __restrict__ best = rs.best;
    const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
    const unsigned count = min(*count_p, cap);
    const unsigned start = start_p ? min(*start_p, cap) : 0u;
    for (int64_t w = start + (int64_t)blockIdx.x * 8 + wib; w < count;
         w += (int64_t)gridDim.x * 8) {
        const uint32_t id = ids[w];
        const int64_t chunk = id / na_pad, a = id % na_pad;
        if (a >= na) {  // warp-uniform: a padded row holds no pair (its slots say so)
            vals[w * 32 + lane] = -CUDART_INF_F;
            pair_ids[w * 32 + lane] = ~0ull;
            continue;
        }
        float x[R];
        const float* xa = plane_a + (int64_t)pts_a[a] * n_pad;
#pragma unroll
        for (int r = 0; r < R; ++r) {
            const int k = r * 32 + lane;
            x[r] = k < n ? xa[k] : 0.f;
        }
        const int64_t b = chunk * 32 + lane;
        const bool ok = b < nb && (!self || b > a);
        // a lane without a pair reads a valid row and discards its value
        const float4* yrow = reinterpret_cast<const float4*>(
            plane_b + (int64_t)pts_b[ok ? b : 0] * n_pad);
        float s = 0.f, c = 0.f;
#pragma unroll
        for (int r0 = 0; r0 < R; r0 += 2) {
            if (r0 * 32 < n) {  // warp-uniform
                // the float4s of slices r0 and r0 + 1 that hold members below n
                float4 q[16];
#pragma unroll
                for (int u = 0; u < 16; ++u) {
                    const int m0 = r0 * 32 + 4 * u;
                    q[u] = (r0 + u / 8 < R && m0 < n) ? __ldg(yrow + r0 * 8 + u)
                                                      : make_float4(0.f, 0.f, 0.f, 0.f);
                }
#pragma unroll
                for (int u = 0; u < 16; ++u) {
                    const int r = r0 + u / 8;
                    if (r < R) {
                        const float yq[4] = {q[u].x, q[u].y, q[u].z, q[u].w};
#pragma unroll
                        for (int e = 0; e < 4; ++e) {
                            const int kk = 4 * (u % 8) + e;  // member r * 32 + kk
                            if (r * 32 + kk < n) {
                                const float xv = __shfl_sync(0xffffffffu, x[r], kk);
                                const float yv = yq[e];
                                const float p = __fmul_rn(xv, yv);
                                const float pe = fmaf(xv, yv, -p);  // TwoProduct error, exact
                                float t, qq;
                                two_sum(s, p, t, qq);
                                s = t;
                                c = __fadd_rn(c, __fadd_rn(qq, pe));
                            }
                        }
                    }
                }
            }
        }
        const float mine = ok ? sign * __fadd_rn(s, c) : -CUDART_INF_F;
        const unsigned long long mine_id = ok ? (unsigned long long)(a * nb + b) : ~0ull;
        vals[w * 32 + lane] = mine;
        pair_ids[w * 32 + lane] = mine_id;
        // best (signed) value, smallest pair index on ties: the warp's maximum
        // key, then one atomic per chunk (one address is shared by all chunks)
        unsigned long long key =
            mine > -CUDART_INF_F
                ? ((unsigned long long)okey(mine) << 32) | (0xffffffffull - (mine_id & 0xffffffffull))
                : 0ull;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            const unsigned long long other = __shfl_xor_sync(0xffffffffu, key, o);
            key = other > key ? other : key;
        }
        if (lane == 0 && key != 0ull) atomicMax(best, key);
    }
}

// For n > 128 (more than four member slices) one warp evaluates the chunk's
// pairs one after another, each with a warp-wide Dot2 (lanes over members,
// compensated tree reduction): the lane-per-pair form would unroll 32 slices
// of 32 loads each.
template <int R>
__global__ void __launch_bounds__(256)
    k_refine_chunks_warp(const float* __restrict__ plane_a, const float* __restrict__ plane_b,
                         int n_pad, int n, const uint32_t* __restrict__ pts_a, int64_t na,
                         const uint32_t* __restrict__ pts_b, int64_t nb, int self,
                         int64_t na_pad, unsigned cap, RefineArgs args) {
    const RefineSide& rs = args.s[blockIdx.y];
    const uint32_t* __restrict__ ids = rs.ids;
    const unsigned* __restrict__ start_p = rs.start;
    const unsigned* __restrict__ count_p = rs.count;
    const float sign = rs.sign;
    float* __restrict__ vals = rs.vals;
    unsigned long long* __restrict__ pair_ids = rs.pair_ids;
    unsigned long long* __restrict__ best = rs.best;
    const int lane = threadIdx.x & 31;
    const unsigned count = min(*count_p, cap);
    const unsigned start = start_p ? min(*start_p, cap) : 0u;
    for (int64_t w = start + (int64_t)blockIdx.x * 8 + (threadIdx.x >> 5); w < count;
         w += (int64_t)gridDim.x * 8) {
        const uint32_t id = ids[w];
        const int64_t chunk = id / na_pad, a = id % na_pad;
        if (a >= na) {  // warp-uniform: a padded row holds no pair (its slots say so)
            vals[w * 32 + lane] = -CUDART_INF_F;
            pair_ids[w * 32 + lane] = ~0ull;
            continue;
        }
        float x[R];
        const float* xa = plane_a + (int64_t)pts_a[a] * n_pad;
#pragma unroll
        for (int r = 0; r < R; ++r) {
            const int k = r * 32 + lane;
            x[r] = k < n ? xa[k] : 0.f;
        }
        float mine = -CUDART_INF_F;
        unsigned long long mine_id = ~0ull;
        for (int j = 0; j < 32; ++j) {
            const int64_t b = chunk * 32 + j;
            const bool ok = b < nb && (!self || b > a);
            float r = -CUDART_INF_F;
            if (ok) r = sign * dot2_warp<R>(x, plane_b + (int64_t)pts_b[b] * n_pad, n);
            if (lane == j) {
                mine = r;
                mine_id = ok ? (unsigned long long)(a * nb + b) : ~0ull;
            }
        }
        vals[w * 32 + lane] = mine;
        pair_ids[w * 32 + lane] = mine_id;
        unsigned long long key =
            mine > -CUDART_INF_F
                ? ((unsigned long long)okey(mine) << 32) | (0xffffffffull - (mine_id & 0xffffffffull))
                : 0ull;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            const unsigned long long other = __shfl_xor_sync(0xffffffffu, key, o);
            key = other > key ? other : key;
        }
        if (lane == 0 && key != 0ull) atomicMax(best, key);
    }
}

// r* - B as a value threshold for the second pass (sign-adjusted domain) of
// each side; records where the first pass's candidates end.
__global__ void k_second_threshold(SideState* ss, int nsides, const unsigned* emax_a,
                                   const unsigned* emax_b, float acc_rel) {
    const float e = fmaxf(__uint_as_float(*emax_a), __uint_as_float(*emax_b));
    const float B = 2.f * e + e * e + (1.f + e) * (1.f + e) * acc_rel + 1e-6f;
    for (int s = 0; s < nsides; ++s) {
        const float rstar = okey_inv((unsigned)(ss[s].best >> 32));
        ss[s].thr[0] = rstar - B;
        ss[s].thr[1] = B;
        ss[s].sel.pass1 = ss[s].sel.count;
    }
}

// 5. top-K of up to 8192 (value, pair) entries taken from the compacted
// refined values, sorted descending. An entry is the 64-bit key
// okey(value) << 32 | (2^32 - 1 - pair id): pair ids are below 2^32, so keys
// are unique, order by value and then by smallest pair id, and give the id
// back. Two kernels:
//   k_topk_chunks  CTA c sorts entries 1024 c .. 1024 c + 1023 (bitonic,
//                  8 per thread: register, shuffle and shared-memory stages)
//                  into scratch, descending, missing entries as key 0;
//   k_topk_rank    every entry's final position is its position in its own
//                  chunk plus, for each other chunk, the number of its keys
//                  that are larger (binary search; keys are unique), and
//                  entries placed below topk are written out.
constexpr int kTopChunk = 1024, kTopMax = 8192;
// keys per thread of k_topk_chunks: 512 threads a chunk, so each SM
// sub-partition holds four warps to hide the exchange latencies
constexpr int kTopE = 2;

template <int D, int E>
__device__ __forceinline__ void sort_regs(unsigned long long (&key)[E], int i0, int size) {
#pragma unroll
    for (int e = 0; e < E; ++e) {
        constexpr int dd = D;
        const int e2 = e ^ dd;
        if (e2 > e) {
            const bool desc = ((i0 + e) & size) == 0;
            const unsigned long long a = key[e], b = key[e2];
            const bool swap = (a < b) == desc;
            key[e] = swap ? b : a;
            key[e2] = swap ? a : b;
        }
    }
}

__global__ void __launch_bounds__(kTopChunk / kTopE)
    k_topk_chunks(const float* __restrict__ vals, const unsigned long long* __restrict__ pids,
                  const uint32_t* __restrict__ sel_idx, const unsigned* __restrict__ count_p,
                  unsigned cap, unsigned long long* __restrict__ sorted) {
    __shared__ unsigned long long skey[kTopChunk];
    constexpr int E = kTopE;
    const int t = threadIdx.x, c0 = blockIdx.x * kTopChunk;
    const unsigned count = min(min(*count_p, cap), (unsigned)kTopMax);
    if ((unsigned)c0 >= count) return;  // block-uniform: an empty chunk is never read
    unsigned long long key[E];
#pragma unroll
    for (int e = 0; e < E; ++e) {
        const unsigned i = (unsigned)(c0 + t * E + e);
        if (i < count) {
            const uint32_t j = sel_idx[i];
            const unsigned long long id = pids ? pids[j] : (unsigned long long)j;
            key[e] = ((unsigned long long)okey(vals[j]) << 32) | (0xffffffffull - (id & 0xffffffffull));
        } else {
            key[e] = 0;
        }
    }
    for (int size = 2; size <= kTopChunk; size <<= 1) {
        for (int d = size >> 1; d > 0; d >>= 1) {
            if (d >= 32 * E) {  // partner in another warp
                __syncthreads();
#pragma unroll
                for (int e = 0; e < E; ++e) skey[t * E + e] = key[e];
                __syncthreads();
#pragma unroll
                for (int e = 0; e < E; ++e) {
                    const int i = t * E + e, q = i ^ d;
                    const unsigned long long o = skey[q];
                    const bool keep_max = (i < q) == ((i & size) == 0);
                    key[e] = (keep_max ? o > key[e] : o < key[e]) ? o : key[e];
                }
            } else if (d >= E) {  // partner lane t ^ (d / E) of the same warp
#pragma unroll
                for (int e = 0; e < E; ++e) {
                    const int i = t * E + e, q = i ^ d;
                    const unsigned long long o = __shfl_xor_sync(0xffffffffu, key[e], d / E);
                    const bool keep_max = (i < q) == ((i & size) == 0);
                    key[e] = (keep_max ? o > key[e] : o < key[e]) ? o : key[e];
                }
            } else if (d == 4) {
                if constexpr (E > 4) sort_regs<4, E>(key, t * E, size);
            } else if (d == 2) {
                if constexpr (E > 2) sort_regs<2, E>(key, t * E, size);
            } else {
                sort_regs<1, E>(key, t * E, size);
            }
        }
    }
#pragma unroll
    for (int e = 0; e < E; ++e) sorted[c0 + t * E + e] = key[e];
}

__global__ void __launch_bounds__(256)
    k_topk_rank(const unsigned long long* __restrict__ sorted, const unsigned* __restrict__ count_p,
                unsigned cap, float sign, int topk, float* __restrict__ out_vals,
                unsigned long long* __restrict__ out_ids) {
    const int g = blockIdx.x * blockDim.x + threadIdx.x;
    const unsigned count = min(min(*count_p, cap), (unsigned)kTopMax);
    const int nchunks = (int)((count + kTopChunk - 1) / kTopChunk);
    if ((unsigned)g >= count) {  // positions past the entries: empty
        if (g < topk) {
            out_vals[g] = -sign * CUDART_INF_F;
            out_ids[g] = ~0ull;
        }
        return;
    }
    const int c = g / kTopChunk;
    const unsigned long long key = sorted[g];  // nonzero: a real entry
    int rank = g - c * kTopChunk;
    for (int o = 0; o < nchunks; ++o) {
        if (o == c) continue;
        // keys of chunk o are descending: count those above key
        const unsigned long long* ch = sorted + o * kTopChunk;
        int lo = 0;
        for (int step = kTopChunk / 2; step > 0; step >>= 1)
            if (ch[lo + step - 1] > key) lo += step;
        rank += lo + (ch[lo] > key ? 1 : 0);
    }
    if (rank < topk) {
        out_vals[rank] = sign * okey_inv((unsigned)(key >> 32));
        out_ids[rank] = 0xffffffffull - (key & 0xffffffffull);
    }
}

// ---------------------------------------------------------------------------
cudaError_t launch_quantize(bool fp8, const float* plane, int n_pad, int n, const uint32_t* pts,
                            int64_t np, int64_t np_pad, int kbytes, void* q, float* inv_scale,
                            unsigned* emax_bits, cudaStream_t st) {
    note_launch();
    const unsigned blocks = (unsigned)((np_pad + 7) / 8);
    if (fp8)
        k_quantize<true><<<blocks, 256, 0, st>>>(plane, n_pad, n, pts, np, np_pad, kbytes,
                                                 (unsigned char*)q, inv_scale, emax_bits);
    else
        k_quantize<false><<<blocks, 256, 0, st>>>(plane, n_pad, n, pts, np, np_pad, kbytes,
                                                  (unsigned char*)q, inv_scale, emax_bits);
    return cudaGetLastError();
}

cudaError_t launch_quantize_ranks(const int16_t* rank2, int n_pad, int n, const uint32_t* pts,
                                  int64_t np, int64_t np_pad, int kbytes, void* q,
                                  float* inv_scale, cudaStream_t st) {
    if (n > 257) return cudaErrorInvalidValue;
    note_launch();
    k_quantize_ranks<<<(unsigned)((np_pad + 7) / 8), 256, 0, st>>>(
        rank2, n_pad, n, pts, np, np_pad, kbytes, (unsigned char*)q, inv_scale);
    return cudaGetLastError();
}

static unsigned grid_for(int64_t N, int per_block) {
    int64_t b = (N + per_block - 1) / per_block;
    if (b < 1) b = 1;
    const int64_t cap = (int64_t)sm_count() * 8;
    if (b > cap) b = cap;
    return (unsigned)b;
}

// Select keys of sign*v into the top `want` (>= want when ties/bins), compact
// their indices into out (capacity cap). scratch: hist[4096] zeroed, sel.
cudaError_t launch_select_top(const float* v, int64_t N, float sign, unsigned want,
                              unsigned* hist, Select* sel, uint32_t* out, unsigned cap,
                              cudaStream_t st, const unsigned* nchunks) {
    SideVals sv{};
    sv.v[0] = sv.v[1] = v;
    sv.sign[0] = sv.sign[1] = sign;
    sv.sel[0] = sv.sel[1] = sel;
    note_launch(5);
    k_hist12<1><<<grid_for(N, 256 * 16), 256, 0, st>>>(sv, N, 0, 20, hist, nchunks);
    k_pick_bin<<<1, 1024, 0, st>>>(hist, 0, 20, want, want, sv);
    k_hist12<1><<<grid_for(N, 256 * 16), 256, 0, st>>>(sv, N, 1, 20, hist, nchunks);
    k_pick_bin<<<1, 1024, 0, st>>>(hist, 1, 20, want, want, sv);
    k_compact<1><<<grid_for(N, 256 * 8), 256, 0, st>>>(sv, N, out, cap, nchunks);
    return cudaGetLastError();
}

static SideVals two_sides(const float* v0, const float* v1, SideState* ss) {
    SideVals sv{};
    sv.v[0] = v0;
    sv.v[1] = v1;
    sv.sign[0] = 1.f;
    sv.sign[1] = -1.f;
    sv.sel[0] = &ss[0].sel;
    sv.sel[1] = &ss[1].sel;
    return sv;
}

cudaError_t launch_select_top2(const float* v0, const float* v1, int64_t N, unsigned want0,
                               unsigned want1, unsigned* hist, bool hist0_built, SideState* ss,
                               uint32_t* out, unsigned cap, cudaStream_t st) {
    if (N % 4) return cudaErrorInvalidValue;
    const SideVals sv = two_sides(v0, v1, ss);
    // the first-level histogram: built by the tensor-core kernel (11 bits), or
    // here (12 bits)
    const int shift = hist0_built ? 21 : 20;
    note_launch(hist0_built ? 4 : 5);
    if (!hist0_built)
        k_hist12<2><<<grid_for(N, 256 * 16), 256, 0, st>>>(sv, N, 0, shift, hist, nullptr);
    k_pick_bin<<<2, 1024, 0, st>>>(hist, 0, shift, want0, want1, sv);
    k_hist12<2><<<grid_for(N, 256 * 16), 256, 0, st>>>(sv, N, 1, shift, hist, nullptr);
    k_pick_bin<<<2, 1024, 0, st>>>(hist, 1, shift, want0, want1, sv);
    k_compact<2><<<grid_for(N, 256 * 8), 256, 0, st>>>(sv, N, out, cap, nullptr);
    return cudaGetLastError();
}

cudaError_t launch_compact_second2(const float* v0, const float* v1, int64_t N, SideState* ss,
                                   uint32_t* out, unsigned cap, cudaStream_t st) {
    if (N % 4) return cudaErrorInvalidValue;
    SideVals sv = two_sides(v0, v1, ss);
    sv.lo_val[0] = &ss[0].thr[0];
    sv.lo_val[1] = &ss[1].thr[0];
    note_launch();
    k_compact<2><<<grid_for(N, 256 * 8), 256, 0, st>>>(sv, N, out, cap, nullptr);
    return cudaGetLastError();
}

cudaError_t launch_refine_chunks2(const float* plane_a, const float* plane_b, int n_pad, int n,
                                  const uint32_t* pts_a, int64_t na, const uint32_t* pts_b,
                                  int64_t nb, int self, int64_t na_pad, const uint32_t* ids,
                                  unsigned cap, SideState* ss, bool first_pass, float* vals,
                                  unsigned long long* pair_ids, bool wide, cudaStream_t st) {
    RefineArgs a{};
    for (int s = 0; s < 2; ++s) {
        a.s[s].ids = ids + (size_t)s * cap;
        a.s[s].start = first_pass ? nullptr : &ss[s].sel.pass1;
        a.s[s].count = &ss[s].sel.count;
        a.s[s].sign = s ? -1.f : 1.f;
        a.s[s].vals = vals + (size_t)s * cap * 32;
        a.s[s].pair_ids = pair_ids + (size_t)s * cap * 32;
        a.s[s].best = &ss[s].best;
    }
    note_launch();
    // blocks per side: a loose bound (wide) refines millions of pairs, often on
    // one side only; a tight one a few thousand chunks, where extra blocks only
    // add scheduling
    const dim3 grid((unsigned)sm_count() * (wide ? 8 : 4), 2);
#define CC_REFINE(K, R)                                                                         \
    K<R><<<grid, 256, 0, st>>>(plane_a, plane_b, n_pad, n, pts_a, na, pts_b, nb, self, na_pad, \
                               cap, a)
    const int slices = (n + 31) / 32;
    if (slices <= 1) CC_REFINE(k_refine_chunks, 1);
    else if (slices <= 2) CC_REFINE(k_refine_chunks, 2);
    else if (slices <= 4) CC_REFINE(k_refine_chunks, 4);
    else if (slices <= 8) CC_REFINE(k_refine_chunks_warp, 8);
    else if (slices <= 16) CC_REFINE(k_refine_chunks_warp, 16);
    else CC_REFINE(k_refine_chunks_warp, 32);
#undef CC_REFINE
    return cudaGetLastError();
}

cudaError_t launch_second_threshold2(SideState* ss, const unsigned* emax_a,
                                     const unsigned* emax_b, float acc_rel, cudaStream_t st) {
    note_launch();
    k_second_threshold<<<1, 1, 0, st>>>(ss, 2, emax_a, emax_b, acc_rel);
    return cudaGetLastError();
}

cudaError_t launch_sort_top(const float* vals, const unsigned long long* pids,
                            const uint32_t* sel_idx, const unsigned* count, unsigned cap,
                            float sign, int topk, float* out_vals, unsigned long long* out_ids,
                            unsigned long long* scratch, cudaStream_t st) {
    if (topk < 0 || topk > kTopMax) return cudaErrorInvalidValue;
    note_launch(2);
    k_topk_chunks<<<kTopMax / kTopChunk, kTopChunk / kTopE, 0, st>>>(vals, pids, sel_idx, count, cap,
                                                                 scratch);
    k_topk_rank<<<kTopMax / 256, 256, 0, st>>>(scratch, count, cap, sign, topk, out_vals,
                                               out_ids);
    return cudaGetLastError();
}

// top-k of vals[sel_idx[i]] where the selected index is itself the id
cudaError_t launch_sort_top_ids(const float* vals, const uint32_t* sel_idx, const unsigned* count,
                                unsigned cap, int topk, float* out_vals,
                                unsigned long long* out_ids, unsigned long long* scratch,
                                cudaStream_t st) {
    return launch_sort_top(vals, nullptr, sel_idx, count, cap, 1.f, topk, out_vals, out_ids,
                           scratch, st);
}

// 3c for a plain pair batch: Dot2 Pearson/Spearman (precision CC_FP32_DOT2).
template <int R>
__global__ void __launch_bounds__(256)
    k_dot2_pairs(const float* __restrict__ A, int64_t Pa, const float* __restrict__ B, int64_t Pb,
                 int n_pad, int n, const uint32_t* __restrict__ pa, const uint32_t* __restrict__ pb,
                 int64_t N, float* __restrict__ out, int* status) {
    const int lane = threadIdx.x & 31;
    for (int64_t t = (int64_t)blockIdx.x * 8 + (threadIdx.x >> 5); t < N;
         t += (int64_t)gridDim.x * 8) {
        const uint32_t p = pa[t], q = pb[t];
        if (p >= Pa || q >= Pb) {
            if (lane == 0) {
                out[t] = CUDART_NAN_F;
                set_status(status, DEV_BAD_INDEX);
            }
            continue;
        }
        float x[R];
        const float* xa = A + (int64_t)p * n_pad;
#pragma unroll
        for (int r = 0; r < R; ++r) {
            const int k = r * 32 + lane;
            x[r] = k < n ? xa[k] : 0.f;
        }
        const float r = dot2_warp<R>(x, B + (int64_t)q * n_pad, n);
        if (lane == 0) out[t] = r;
    }
}

cudaError_t launch_dot2_pairs(const float* A, int64_t Pa, const float* B, int64_t Pb, int n_pad,
                              int n, const uint32_t* pa, const uint32_t* pb, int64_t N, float* out,
                              int* status, cudaStream_t st) {
    if (N <= 0) return cudaSuccess;
    note_launch();
#define CC_DOT2(R) \
    k_dot2_pairs<R><<<grid_for(N, 8), 256, 0, st>>>(A, Pa, B, Pb, n_pad, n, pa, pb, N, out, status)
    const int slices = (n + 31) / 32;
    if (slices <= 1) CC_DOT2(1);
    else if (slices <= 2) CC_DOT2(2);
    else if (slices <= 4) CC_DOT2(4);
    else if (slices <= 8) CC_DOT2(8);
    else if (slices <= 16) CC_DOT2(16);
    else CC_DOT2(32);
#undef CC_DOT2
    return cudaGetLastError();
}

}  // namespace cc
