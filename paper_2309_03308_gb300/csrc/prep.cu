// Field ingest and per-point planes (Section 3: an ensemble of n members on
// a 3D grid; Section 3.2: PPMCC needs only means and variances, KSG needs the
// per-sample neighbour structure, binned MI needs per-point bins).
//
// Every plane is point-major [P][n_pad] so a pair kernel reads each point's
// member vector as one contiguous, aligned row.
#include "device.cuh"
#include "internal.cuh"

namespace cc {

// ----------------------------------------------------------------------------
// [n][P] member-major input -> [P][n_pad] point-major values. A CTA moves 32
// points x all members through a shared-memory tile: every row of 32 input
// floats is one coalesced 128-byte read (a thread keeps up to 16 in flight),
// every point row is written as coalesced float4 stores. Padding members are
// 0. Non-finite inputs set DEV_NONFINITE.
constexpr int kIngestPts = 32;

__global__ void __launch_bounds__(256)
    k_ingest(const float* __restrict__ in, int n, int64_t P, int64_t in_stride, int n_pad,
             float* __restrict__ vals, int* status) {
    extern __shared__ float tile[];  // [n_pad][kIngestPts + 1]
    const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;
    const int64_t p0 = (int64_t)blockIdx.x * kIngestPts;
    const int64_t p = p0 + tx;
    bool bad = false;
    for (int m0 = 0; m0 < n_pad; m0 += 8 * 16) {
        float v[16];
#pragma unroll
        for (int u = 0; u < 16; ++u) {
            const int m = m0 + 8 * u + ty;
            v[u] = (m < n && p < P) ? __ldcs(in + (int64_t)m * in_stride + p) : 0.f;
        }
#pragma unroll
        for (int u = 0; u < 16; ++u) {
            const int m = m0 + 8 * u + ty;
            bad |= !isfinite(v[u]);
            if (m < n_pad) tile[m * (kIngestPts + 1) + tx] = v[u];
        }
    }
    if (bad) set_status(status, DEV_NONFINITE);
    __syncthreads();
    const int q = n_pad / 4;  // float4 per point row
    for (int e = threadIdx.x; e < kIngestPts * q; e += blockDim.x) {
        const int pt = e / q, m = 4 * (e % q);
        if (p0 + pt >= P) continue;
        const float4 o = make_float4(tile[m * (kIngestPts + 1) + pt],
                                     tile[(m + 1) * (kIngestPts + 1) + pt],
                                     tile[(m + 2) * (kIngestPts + 1) + pt],
                                     tile[(m + 3) * (kIngestPts + 1) + pt]);
        *reinterpret_cast<float4*>(vals + (p0 + pt) * n_pad + m) = o;
    }
}

cudaError_t launch_ingest(const float* in, int n, int64_t P, int64_t in_stride, int n_pad,
                          float* vals, int* status, cudaStream_t st) {
    const size_t smem = sizeof(float) * (size_t)n_pad * (kIngestPts + 1);
    if (smem > 48 * 1024) {
        cudaError_t e =
            cudaFuncSetAttribute(k_ingest, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
    }
    note_launch();
    k_ingest<<<(unsigned)((P + kIngestPts - 1) / kIngestPts), 256, smem, st>>>(
        in, n, P, in_stride, n_pad, vals, status);
    return cudaGetLastError();
}

// ----------------------------------------------------------------------------
// One warp per grid point, member vector in registers in blocked layout
// (lane l holds members l*E .. l*E+E-1, E = n_pad / 32):
//   mean, ss      sum, then sum of squared deviations about the mean, each
//                 accumulated in float-float (TwoSum / exact FMA products, ~2^-44
//                 relative) and finalised in FP64 (the per-point FP64 work is a
//                 few instructions: this GPU's FP64 rate is a small fraction of
//                 its FP32 rate)
//   zhat          (v - mean) / sqrt(ss) rounded to fp32 (0 when ss == 0); the
//                 scale 1 / sqrt(ss) by a float-float Newton step (ff_rsqrt)
//   sorted, perm  ascending order, stable: a warp bitonic sort of the unique
//                 64-bit keys (order-preserving bits of v + 0.0f, member index),
//                 so -0.0 and +0.0 tie and equal values keep member order. For
//                 n_pad <= 128 the warp first sorts 32-bit keys (the top 25
//                 order bits, the 7-bit member index): the same order whenever
//                 no two members share those 25 bits (values within 2^7 ulp of
//                 each other, ties included), which the warp checks on adjacent
//                 sorted keys, taking the 64-bit sort otherwise
//   rank2         2 * average rank (ties averaged): for a run of equal values
//                 at sorted positions a..b, every member gets a + b + 2
//                 (= 2L + E + 1 with L values below and E equal)
//   rhat          c / sqrt(sum c^2) with c = rank2 - (n + 1) (exact integers)
constexpr int kPrepWarps = 4;

__device__ __forceinline__ unsigned order_bits(float v) {
    const unsigned b = __float_as_uint(v + 0.0f);  // -0.0 -> +0.0
    return (b & 0x80000000u) ? ~b : (b | 0x80000000u);
}
__device__ __forceinline__ float unorder_bits(unsigned o) {
    return __uint_as_float((o & 0x80000000u) ? (o & 0x7fffffffu) : ~o);
}

// 1 / sqrt(h + l) rounded to fp32, for a float-float h + l with h > 0 and
// |l| <= ulp(h) / 2: the hardware estimate y (relative error e0 ~ 2^-22) and
// one Newton step y (1 + e / 2 + 3 e^2 / 8) on the residual e = 1 - (h + l) y^2,
// which is formed from exact FMA products (absolute error ~2^-44). The value
// before the final rounding is within ~2^-43 of 1 / sqrt(h + l), so the result
// is the correctly rounded one except within that distance of a rounding
// boundary. FP32 pipe only: a warp-wide FP64 instruction holds GB300's narrow
// FP64 pipe for many cycles.
__device__ __forceinline__ float ff_rsqrt(float h, float l) {
    const float y = rsqrtf(h);
    const float yy = __fmul_rn(y, y);
    const float yy_l = fmaf(y, y, -yy);  // y^2 = yy + yy_l exactly
    float e = fmaf(-h, yy, 1.0f);        // 1 - h yy, the product exact
    e = fmaf(-h, yy_l, e);
    e = fmaf(-l, yy, e);
    const float t = fmaf(0.375f * e, e, 0.5f * e);
    return fmaf(y, t, y);
}

// warp maximum of non-negative floats: their bit patterns order as integers
__device__ __forceinline__ float warp_max_f32(float v) {
    return __uint_as_float(__reduce_max_sync(0xffffffffu, __float_as_uint(v)));
}

// power of two s with m * s in [1, 2) for finite normal m > 0 (1 for m == 0)
__device__ __forceinline__ float pow2_scale(float m) {
    if (!(m > 0.f)) return 1.f;
    int ex;
    frexpf(m, &ex);  // m = f * 2^ex, f in [0.5, 1)
    return ldexpf(1.f, min(1 - ex, 126));  // below 2^-126 (subnormal m): 2^126
}

// Ascending warp bitonic sort of 32 * E unique keys, lane l holding positions
// l*E .. l*E+E-1. Exchange across lanes: the element takes its partner's key
// when (partner < own) equals "this element keeps the minimum", one
// comparison; the keep-minimum flag depends on the lane only, since
// e < E <= d leaves the bits d and size of g0 + e to g0.
template <int E, class K>
__device__ __forceinline__ void warp_bitonic(K (&key)[E], int g0) {
    constexpr int NP = 32 * E;
#pragma unroll
    for (int size = 2; size <= NP; size <<= 1) {
#pragma unroll
        for (int d = size >> 1; d > 0; d >>= 1) {
            if (d >= E) {
                const bool keep_min = ((g0 & d) == 0) == ((g0 & size) == 0);
#pragma unroll
                for (int e = 0; e < E; ++e) {
                    const K o = __shfl_xor_sync(0xffffffffu, key[e], d / E);
                    key[e] = ((o < key[e]) == keep_min) ? o : key[e];
                }
            } else {
#pragma unroll
                for (int e = 0; e < E; ++e) {
                    const int e2 = e ^ d;
                    if (e2 > e) {
                        const bool asc = ((g0 + e) & size) == 0;
                        const bool swap = (key[e2] < key[e]) == asc;
                        const K a = key[e], b = key[e2];
                        key[e] = swap ? b : a;
                        key[e2] = swap ? a : b;
                    }
                }
            }
        }
    }
}

// resident blocks per SM the register allocation must allow (E = 4: the
// n <= 128 workloads, 9 blocks of 4 warps at <= 56 registers)
__host__ __device__ constexpr int prep_min_blocks(int E) {
    return E == 1 ? 12 : E == 2 ? 10 : E == 4 ? 9 : E == 8 ? 6 : E == 16 ? 4 : 3;
}

template <int E>
__global__ void __launch_bounds__(kPrepWarps * 32, prep_min_blocks(E))
    k_point_prep(const float* __restrict__ vals, int64_t p_begin, int64_t P, int n, float nf,
                 float* __restrict__ sorted,
                 uint16_t* __restrict__ perm, int16_t* __restrict__ rank2,
                 float* __restrict__ zhat, float* __restrict__ rhat,
                 double* __restrict__ mean_out, double* __restrict__ ss_out, PrepBins pb) {
    __shared__ int bin_hist[kPrepWarps][16];
    constexpr int NP = 32 * E;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int64_t p = p_begin + (int64_t)blockIdx.x * kPrepWarps + warp;
    if (p >= P) return;
    const int64_t row = p * NP;
    const int g0 = lane * E;

    unsigned long long key[E];
    float dev[E];  // v - mean rounded to fp32, times 2^-ed; scaled to z below
    float ss_h = 0.f, ss_l = 0.f;
    float mean_h, mean_l, vscale, dscale;
    {
        float v[E];
#pragma unroll
        for (int e = 0; e < E; ++e) v[e] = vals[row + g0 + e];
#pragma unroll
        for (int e = 0; e < E; ++e)
            key[e] = g0 + e < n ? ((unsigned long long)order_bits(v[e]) << 32) | (unsigned)(g0 + e)
                                : (0xffffffffull << 32) | (unsigned)(g0 + e);
        // exact power-of-two scaling to max |v| in [1, 2): the float-float
        // sums below neither overflow nor lose their low parts to underflow
        float mv = 0.f;
#pragma unroll
        for (int e = 0; e < E; ++e)
            if (g0 + e < n) mv = fmaxf(mv, fabsf(v[e]));
        vscale = pow2_scale(warp_max_f32(mv));
        // sum in float-float (error-free transformations; ~2^-44 relative)
        float sh = 0.f, sl = 0.f;
#pragma unroll
        for (int e = 0; e < E; ++e) {
            v[e] *= vscale;
            if (g0 + e < n) ff_add(sh, sl, v[e], 0.f);
        }
        warp_sum_ff(sh, sl);
        // mean = (sh + sl) / n as mean_h + mean_l: the remainder of a rounded
        // quotient is exact under FMA
        mean_h = __fdiv_rn(sh, nf);
        const float rem = __fadd_rn(fmaf(-mean_h, nf, sh), sl);
        mean_l = __fdiv_rn(rem, nf);
        // deviations dh + dl = v - mean (TwoSum; dh is v - mean rounded)
        float dl[E], md = 0.f;
#pragma unroll
        for (int e = 0; e < E; ++e) {
            float a, ea;
            two_sum(v[e], -mean_h, a, ea);
            two_sum(a, __fsub_rn(ea, mean_l), dev[e], dl[e]);
            if (g0 + e < n) md = fmaxf(md, fabsf(dev[e]));
        }
        // second exact scaling, max |dh| in [1, 2), then the sum of squares
        // in float-float (exact products, the dl term to first order)
        dscale = pow2_scale(warp_max_f32(md));
#pragma unroll
        for (int e = 0; e < E; ++e) {
            const float dh = dev[e] * dscale, dle = dl[e] * dscale;
            dev[e] = dh;
            if (g0 + e < n) {
                const float p = __fmul_rn(dh, dh);
                const float pe = fmaf(dh, dh, -p) + 2.f * dh * dle;
                ff_add(ss_h, ss_l, p, pe);
            }
        }
        warp_sum_ff(ss_h, ss_l);
    }

    // ascending sort of the unique 64-bit keys
    bool sorted32 = false;
    if constexpr (NP <= 128) {
        unsigned k32[E];
#pragma unroll
        for (int e = 0; e < E; ++e)
            k32[e] = ((unsigned)(key[e] >> 32) & 0xffffff80u) | (unsigned)(g0 + e);
        warp_bitonic<E>(k32, g0);
        // the 64-bit keys' order unless two real members share the top 25
        // bits; such members are adjacent in it
        const unsigned next = __shfl_down_sync(0xffffffffu, k32[0], 1);
        bool clash = false;
#pragma unroll
        for (int e = 0; e < E; ++e) {
            const unsigned nk = e + 1 < E ? k32[e + 1] : next;
            clash |= g0 + e + 1 < n && (nk >> 7) == (k32[e] >> 7);
        }
        if (!__any_sync(0xffffffffu, clash)) {  // the sorted 64-bit keys, rebuilt
#pragma unroll
            for (int e = 0; e < E; ++e) {
                const unsigned m = k32[e] & 0x7fu;
                const unsigned hi = g0 + e < n ? order_bits(vals[row + m]) : 0xffffffffu;
                key[e] = ((unsigned long long)hi << 32) | m;
            }
            sorted32 = true;
        }
    }
    if (!sorted32) warp_bitonic<E>(key, g0);

    // sorted values, permutation, and runs of equal values
    float sv[E];
#pragma unroll
    for (int e = 0; e < E; ++e) {
        const int g = g0 + e;
        sv[e] = unorder_bits((unsigned)(key[e] >> 32));
        sorted[row + g] = g < n ? sv[e] : CUDART_INF_F;
        perm[row + g] = (uint16_t)(key[e] & 0xffffu);
    }
    // bin planes of the requested bin counts (same fp32 steps as k_bins)
    if (pb.count > 0) {
        __syncwarp();  // the sorted row written above is visible to the warp
        const float lo = sorted[row], hi = sorted[row + n - 1];
        const bool flat = !(hi > lo);
        const float w = __fsub_rn(hi, lo);
        float vm[E];
#pragma unroll
        for (int e = 0; e < E; ++e) vm[e] = vals[row + g0 + e];
        int* hh = bin_hist[warp];
        auto build = [&](const int B, uint8_t* brow, long long* hmarg) {
            if (lane < 16) hh[lane] = 0;
            __syncwarp();
            uint32_t word = 0;
#pragma unroll
            for (int e = 0; e < E; ++e) {
                const int g = g0 + e;
                int b = 0;
                if (g < n && !flat) {
                    const float t = __fsub_rn(vm[e], lo);
                    const float r = __fdiv_rn(t, w);
                    const float sc = __fmul_rn(r, (float)B);
                    b = (int)floorf(sc);
                    b = b < 0 ? 0 : (b > B - 1 ? B - 1 : b);
                }
                if (g < n) atomicAdd(&hh[b], 1);
                if (E % 4 == 0) {
                    word |= (uint32_t)b << (8 * (e & 3));
                    if ((e & 3) == 3) {
                        *reinterpret_cast<uint32_t*>(brow + g - 3) = word;
                        word = 0;
                    }
                } else {
                    brow[g] = (uint8_t)b;
                }
            }
            __syncwarp();
            long long sm = lane < B ? pb.clogc[hh[lane]] : 0;
            sm = warp_sum_u64_redux(sm);  // c ln c >= 0
            if (lane == 0) hmarg[p] = sm;
            __syncwarp();
        };
        build(pb.B[0], pb.bins[0] + row, pb.hmarg[0]);
        if (pb.count > 1) build(pb.B[1], pb.bins[1] + row, pb.hmarg[1]);
    }
    int r2[E];
    long long c2 = 0;
    if (sorted32) {
        // every value is distinct: the member at sorted position g has
        // rank2 = 2g + 2, and the centred ranks 2g + 1 - n square-sum to
        // n (n^2 - 1) / 3
#pragma unroll
        for (int e = 0; e < E; ++e) r2[e] = 2 * (g0 + e) + 2;
        c2 = (long long)n * ((long long)n * n - 1) / 3;
    } else {
        // run start a: prefix max of (start ? g : 0); run end b: suffix min of (end ? g : NP)
        const float prev_last = __shfl_up_sync(0xffffffffu, sv[E - 1], 1);
        const float next_first = __shfl_down_sync(0xffffffffu, sv[0], 1);
        int a[E], b[E];
#pragma unroll
        for (int e = 0; e < E; ++e) {
            const int g = g0 + e;
            const float pv = e > 0 ? sv[e - 1] : prev_last;
            const bool start = g == 0 || g >= n || !(pv == sv[e]);
            a[e] = start ? g : 0;
            if (e > 0) a[e] = max(a[e], a[e - 1]);
        }
#pragma unroll
        for (int e = E - 1; e >= 0; --e) {
            const int g = g0 + e;
            const float nv = e < E - 1 ? sv[e + 1] : next_first;
            const bool end = g >= n - 1 || !(nv == sv[e]);
            b[e] = end ? g : NP;
            if (e < E - 1) b[e] = min(b[e], b[e + 1]);
        }
        int carry_a = a[E - 1], carry_b = b[0];
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int ta = __shfl_up_sync(0xffffffffu, carry_a, o);
            const int tb = __shfl_down_sync(0xffffffffu, carry_b, o);
            if (lane >= o) carry_a = max(carry_a, ta);
            if (lane + o < 32) carry_b = min(carry_b, tb);
        }
        const int before_a = __shfl_up_sync(0xffffffffu, carry_a, 1);
        const int after_b = __shfl_down_sync(0xffffffffu, carry_b, 1);
#pragma unroll
        for (int e = 0; e < E; ++e) {
            const int g = g0 + e;
            const int aa = lane > 0 ? max(a[e], before_a) : a[e];
            const int bb = lane < 31 ? min(b[e], after_b) : b[e];
            r2[e] = aa + bb + 2;
            if (g < n) {
                const long long c = r2[e] - (n + 1);
                c2 += c * c;
            }
        }
        // each c^2 <= n^2 <= 2^20 and n <= 1024 values: the sum fits 32 bits
        c2 = (long long)__reduce_add_sync(0xffffffffu, (unsigned)c2);
    }
    // the two norms' reciprocal square roots on the FP32 pipe (the sums are
    // the same on every lane; c2 < 2^29 splits exactly into two floats)
    const float inv = ss_h > 0.f ? ff_rsqrt(ss_h, ss_l) : 0.f;
    const float c2h = (float)c2;
    const float rinv = c2 > 0 ? ff_rsqrt(c2h, (float)(c2 - (long long)c2h)) : 0.f;
    if (lane == 0) {  // FP64 statistics; undo the power-of-two scalings (exact reciprocals)
        const double ss_s = (double)ss_h + (double)ss_l;  // in units of (vscale dscale)^2
        const double rv = (double)__frcp_rn(vscale), rs = rv * (double)__frcp_rn(dscale);
        mean_out[p] = ((double)mean_h + (double)mean_l) * rv;
        ss_out[p] = ss_s * (rs * rs);
    }
#pragma unroll
    for (int e = 0; e < E; ++e) {
        const int g = g0 + e;
        zhat[row + g] = g < n ? dev[e] * inv : 0.f;  // fp32 scale (<= 3 roundings)
    }
#pragma unroll
    for (int e = 0; e < E; ++e) {
        const int g = g0 + e;
        const int m = (int)(key[e] & 0xffffu);  // member at sorted position g
        if (g < n) {
            rank2[row + m] = (int16_t)r2[e];
            rhat[row + m] = (float)(r2[e] - (n + 1)) * rinv;  // exact integer times fp32 scale
        } else {
            rank2[row + g] = 0;
            rhat[row + g] = 0.f;
        }
    }
}

cudaError_t launch_point_prep(const Field& f, cudaStream_t st, const PrepBins& pb,
                              int64_t p_begin, int64_t p_end) {
    if (p_end < 0) p_end = f.P;
    if (p_end <= p_begin) return cudaSuccess;
    const unsigned blocks = (unsigned)((p_end - p_begin + kPrepWarps - 1) / kPrepWarps);
    note_launch();
#define CC_PREP(E)                                                                               \
    k_point_prep<E><<<blocks, kPrepWarps * 32, 0, st>>>(                                         \
        f.vals.as<float>(), p_begin, p_end, f.n, (float)f.n, f.sorted.as<float>(),               \
        f.perm.as<uint16_t>(),                                                                   \
        f.rank2.as<int16_t>(), f.zhat.as<float>(), f.rhat.as<float>(), f.mean.as<double>(),      \
        f.ss.as<double>(), pb)
    switch (f.n_pad / 32) {  // n_pad is a power of two >= 32
        case 1: CC_PREP(1); break;
        case 2: CC_PREP(2); break;
        case 4: CC_PREP(4); break;
        case 8: CC_PREP(8); break;
        case 16: CC_PREP(16); break;
        case 32: CC_PREP(32); break;
        default: return cudaErrorInvalidValue;
    }
#undef CC_PREP
    return cudaGetLastError();
}

// ----------------------------------------------------------------------------
// Spatial aggregate (Section 3.3): one warp per block of the source grid,
// lanes over members (coalesced point rows); mean (FP64 sum, rounded once)
// or maximum per block and member, written member-major [n][Pc].
__global__ void __launch_bounds__(256)
    k_aggregate(const float* __restrict__ vals, int X, int Y, int Z, int n, int n_pad, int bx,
                int by, int bz, int Xc, int Yc, int64_t Pc, int mode, float* __restrict__ out) {
    const int lane = threadIdx.x & 31;
    const int64_t c = (int64_t)blockIdx.x * 8 + (threadIdx.x >> 5);
    if (c >= Pc) return;
    const int ci = (int)(c % Xc), cj = (int)((c / Xc) % Yc), ck = (int)(c / ((int64_t)Xc * Yc));
    const int x0 = ci * bx, y0 = cj * by, z0 = ck * bz;
    const int x1 = min(x0 + bx, X), y1 = min(y0 + by, Y), z1 = min(z0 + bz, Z);
    const double cnt = (double)(x1 - x0) * (y1 - y0) * (z1 - z0);
    for (int m = lane; m < n; m += 32) {
        double s = 0.0;
        float mx = -CUDART_INF_F;
        for (int z = z0; z < z1; ++z)
            for (int y = y0; y < y1; ++y)
                for (int x = x0; x < x1; ++x) {
                    const float v = vals[((int64_t)x + (int64_t)X * (y + (int64_t)Y * z)) * n_pad + m];
                    s += (double)v;
                    mx = fmaxf(mx, v);
                }
        out[(int64_t)m * Pc + c] = mode == 0 ? (float)(s / cnt) : mx;
    }
}

cudaError_t launch_aggregate(const Field& f, int bx, int by, int bz, int Xc, int Yc, int64_t Pc,
                             int mode, float* out, cudaStream_t st) {
    note_launch();
    k_aggregate<<<(unsigned)((Pc + 7) / 8), 256, 0, st>>>(f.vals.as<float>(), f.X, f.Y, f.Z, f.n,
                                                         f.n_pad, bx, by, bz, Xc, Yc, Pc, mode,
                                                         out);
    return cudaGetLastError();
}

// ----------------------------------------------------------------------------
// Bins for B bins per variable (Section 3.2, binning): over the point's own
// [lo, hi] = [min, max], b = floor(((v - lo) / (hi - lo)) * B) with each step
// an IEEE fp32 operation, clamped to [0, B-1]; hi == lo gives bin 0.
// Also the marginal term sum_b c_b ln c_b of the point (fixed point, 2^-40).
__global__ void __launch_bounds__(128)
    k_bins(const float* __restrict__ vals, const float* __restrict__ sorted, int64_t P, int n,
           int n_pad, int B, const long long* __restrict__ clogc_fix, uint8_t* __restrict__ bins,
           long long* __restrict__ hmarg) {
    __shared__ int hist[4][16];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int64_t p = (int64_t)blockIdx.x * 4 + warp;
    if (p >= P) return;
    if (lane < 16) hist[warp][lane] = 0;
    __syncwarp();
    const float lo = sorted[p * n_pad];
    const float hi = sorted[p * n_pad + n - 1];
    const bool flat = !(hi > lo);
    const float w = __fsub_rn(hi, lo);
    // four members per lane per 128-member slice: one float4 in, one word out
    for (int m = 4 * lane; m < n_pad; m += 128) {
        const float4 v4 = *reinterpret_cast<const float4*>(vals + p * n_pad + m);
        const float v[4] = {v4.x, v4.y, v4.z, v4.w};
        uint32_t word = 0;
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            int b = 0;
            if (m + j < n && !flat) {
                const float t = __fsub_rn(v[j], lo);
                const float r = __fdiv_rn(t, w);
                const float sc = __fmul_rn(r, (float)B);
                b = (int)floorf(sc);
                b = b < 0 ? 0 : (b > B - 1 ? B - 1 : b);
            }
            word |= (uint32_t)b << (8 * j);
            if (m + j < n) atomicAdd(&hist[warp][b], 1);
        }
        *reinterpret_cast<uint32_t*>(bins + p * n_pad + m) = word;
    }
    __syncwarp();
    long long s = lane < B ? clogc_fix[hist[warp][lane]] : 0;
    s = warp_sum_u64_redux(s);  // c ln c >= 0
    if (lane == 0) hmarg[p] = s;
}

cudaError_t launch_bins(const Field& f, int B, const int64_t* clogc_fix, uint8_t* bins,
                        int64_t* hmarg, cudaStream_t st) {
    const unsigned blocks = (unsigned)((f.P + 3) / 4);
    note_launch();
    k_bins<<<blocks, 128, 0, st>>>(f.vals.as<float>(), f.sorted.as<float>(), f.P, f.n, f.n_pad,
                                   B, (const long long*)clogc_fix, bins, (long long*)hmarg);
    return cudaGetLastError();
}

// ----------------------------------------------------------------------------
// Member-major compact planes of a region for the all-pairs contraction:
// zT[k][a] = zhat[pts[a]][k] for k < n, a < np; zero elsewhere (k < nk,
// a < np_pad). Same for the rank plane.
__global__ void k_region_planes(const float* __restrict__ zhat, const float* __restrict__ rhat,
                                int n, int n_pad, const uint32_t* __restrict__ pts, int64_t np,
                                int nk, int64_t np_pad, float* __restrict__ zT,
                                float* __restrict__ rT) {
    __shared__ float tz[32][33], tr[32][33];
    const int64_t a0 = (int64_t)blockIdx.x * 32;
    const int k0 = blockIdx.y * 32;
    for (int r = threadIdx.y; r < 32; r += 8) {
        const int64_t a = a0 + r;
        const int k = k0 + threadIdx.x;
        float z = 0.f, q = 0.f;
        if (a < np && k < n) {
            const int64_t off = (int64_t)pts[a] * n_pad + k;
            z = zhat[off];
            q = rhat[off];
        }
        tz[r][threadIdx.x] = z;
        tr[r][threadIdx.x] = q;
    }
    __syncthreads();
    for (int r = threadIdx.y; r < 32; r += 8) {
        const int k = k0 + r;
        const int64_t a = a0 + threadIdx.x;
        if (k < nk && a < np_pad) {
            zT[(int64_t)k * np_pad + a] = tz[threadIdx.x][r];
            rT[(int64_t)k * np_pad + a] = tr[threadIdx.x][r];
        }
    }
}

cudaError_t launch_region_planes(const Field& f, const Region& r, cudaStream_t st) {
    dim3 grid((unsigned)(r.np_pad / 32), (unsigned)((r.nk + 31) / 32));
    note_launch();
    k_region_planes<<<grid, dim3(32, 8), 0, st>>>(f.zhat.as<float>(), f.rhat.as<float>(), f.n,
                                                  f.n_pad, r.pts.as<uint32_t>(), r.np, r.nk,
                                                  r.np_pad, r.zT.as<float>(), r.rT.as<float>());
    return cudaGetLastError();
}

}  // namespace cc
