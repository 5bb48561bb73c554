// Bayesian optimal sampling of brick-pair maxima, batched over all region
// pairs (Section 3.1; Section 6: UCB with kappa = 0.5). One round:
//
//   propose    per region pair, UCB mu + kappa * sigma over a fixed seeded pool
//              of Q continuous 6D positions; the top-M form a shortlist whose
//              posterior covariance is built, and R proposals are picked
//              greedily with the kriging-believer update
//              (cov -= cov[:, c] cov[c, :] / (cov[c, c] + noise)).
//   round      probabilistic reparameterization: voxel = floor(theta) +
//              Bernoulli(theta - floor(theta)) (Philox4x64-10).
//   evaluate   Pearson, Spearman, binned MI and KSG for every (pair, proposal)
//              in ONE persistent launch: warps pull (measure, pair) items from a
//              work queue, longest measure (KSG) first.
//   extremes   running max / min per region pair and measure.
//   condition  the GP of each region pair absorbs the R new observations of the
//              objective measure. The state keeps V = L^-1 K(X, pool) (L the
//              Cholesky factor over the observations X), so conditioning needs
//              only the new rows V2 = L22^-1 (K(P, pool) - V[:, P]^T V) with
//              L22 = chol(posterior cov(P, P) + noise): mean and variance of all
//              pool entries then update as mu += V2^T beta2, var -= colsum(V2^2).
//
// The two contractions of the GP, the shortlist's V[:, SL]^T V[:, SL] and the
// conditioning's V[:, P]^T V, run on the tensor cores in TF32 with each FP32
// operand split exactly into a TF32 head and tail (three products per K step,
// FP32 accumulation in TMEM), which keeps FP32-level accuracy in the
// posterior's cancellation K - V^T V.
//
// Matern nu = 5/2 kernel with ARD length scales 0.25 x extent (voxels); the
// signal variance is the variance of the first round's objective values, the
// noise variance 1e-4 of it, the prior mean their mean (or a supplied value
// per pool entry, e.g. a learned surrogate's prediction). The whole round is
// captured once into a CUDA graph and replayed; kernels read the round number
// from device memory. The evaluation kernel's launch shape is autotuned.
#include <math.h>
#include <stdarg.h>
#include <stdio.h>
#include <stdlib.h>
#include <string.h>

#include <algorithm>
#include <fstream>
#include <mutex>
#include <sstream>
#include <string>
#include <vector>

#include "internal.cuh"
#include "ksg_dev.cuh"
#include "tc_dev.cuh"

namespace cc {

double digamma_int_host(int m);

constexpr uint64_t kPoolKey = 0xB05B05ull, kRoundKey = 0xB0517Dull;
constexpr int kBosThreads = 256;
constexpr int kGRows = 512;  // rows of V[:, P] the conditioning keeps in shared memory
constexpr int kEvalChunk = 8;  // KSG candidates per work-queue pull
// the conditioning's first shared region: G (kGRows x 32 floats), later the
// product's operand stage (40 KB) and its two-block load ring (40 KB)
constexpr size_t kCondRegion0 = 81920;
static_assert(kCondRegion0 >= (size_t)kGRows * 32 * 4, "G fits the first region");

struct BosDev {
    int n_rp, Q, R, T, M;
    int L;        // local proposals per round from the second round on (0: none)
    float lscale; // their spread per axis as a fraction of the region extent
    int S;        // GP observations provisioned: R + (T - 1) (R - L)
    int Sp;       // S rounded up to 8: the stride of one pool entry's column of V
    float kappa;
    uint64_t seed;
    int objective, k, bins;
    int n, n_pad, X, Y;
    const int* box;      // [n_rp][12]: a.x0 y0 z0 ext_x ext_y ext_z, b likewise
    const int* self;     // [n_rp]
    float* pool;         // [n_rp][Q][6]
    float* V;            // [n_rp][Q][Sp] pool-major: column c (observations 0..) contiguous,
                         // zero beyond the rows written so far
    float* mu;           // [n_rp][Q]
    float* var;          // [n_rp][Q]
    unsigned* sel;       // [n_rp][Q/32]
    int* obs;            // [n_rp][R*T]
    float* y;            // [n_rp][R*T]
    float* beta;         // [n_rp][R*T]
    float* hyp;          // [n_rp][4]: prior mean, signal var, noise var
    float* theta;        // [n_rp][R*T][6] every evaluated proposal's position, in order
    float* yall;         // [n_rp][R*T] its objective value
    float* inc_val;      // [n_rp][2] the two best objective values so far
    int* inc_idx;        // [n_rp][2] their sample indices (into theta)
    const float* prior;  // [n_rp][Q] or null
    int* picks;          // [n_rp][R]
    uint32_t* pa;        // [n_rp*R]
    uint32_t* pb;
    float* vals;         // [4][n_rp*R]
    Partial* best;       // [4][n_rp], argmax/argmin = (pa << 32) | pb
    int* round;
    int* queue;          // [2]: next item of the non-KSG measures, next KSG chunk
    int* status;
    // field planes
    const float* zhat;  // planes of the field of the first regions ...
    const float* rhat;
    const float* fvals;
    const float* sorted;
    const uint16_t* perm;
    const uint8_t* bins_p;
    const long long* hmarg;
    const float* zhat_b;  // ... and of the second regions (the same field, or a second
    const float* rhat_b;  // variable on the same grid: Section 4.3)
    const float* fvals_b;
    const float* sorted_b;
    const uint16_t* perm_b;
    const uint8_t* bins_b;
    const long long* hmarg_b;
    const long long* psi_fix;
    const long long* clogc_fix;
    double psi_nk;
    double fix_over_n;  // 1 / (2^40 n): fixed-point sum -> mean
    double logn;
};

// GP observations before round r (round 0 conditions all R proposals, later
// rounds the R - L pool proposals) and new ones in round r
__host__ __device__ __forceinline__ int obs_before(int r, int R, int L) {
    return r == 0 ? 0 : R + (r - 1) * (R - L);
}
__host__ __device__ __forceinline__ int obs_new(int r, int R, int L) { return r == 0 ? R : R - L; }

__device__ __forceinline__ unsigned okey32(float v) {
    const unsigned b = __float_as_uint(v + 0.0f);
    return (b & 0x80000000u) ? ~b : (b | 0x80000000u);
}

__device__ __forceinline__ float matern52(const float* a, const float* b, const float* inv_ell,
                                          float sf2) {
    float r2 = 0.f;
#pragma unroll
    for (int d = 0; d < 6; ++d) {
        const float t = (a[d] - b[d]) * inv_ell[d];
        r2 = fmaf(t, t, r2);
    }
    const float r = sqrtf(r2) * 2.2360679774997896f;  // sqrt(5) r
    return sf2 * (1.f + r + r * r * (1.f / 3.f)) * expf(-r);
}

__device__ __forceinline__ void inv_ell_of(const BosDev& d, int rp, float* inv_ell) {
#pragma unroll
    for (int a = 0; a < 2; ++a)
#pragma unroll
        for (int j = 0; j < 3; ++j) inv_ell[3 * a + j] = 1.f / (0.25f * (float)d.box[rp * 12 + 6 * a + 3 + j]);
}

// ---------------------------------------------------------------------------
// pool: candidate c of pair rp from Philox blocks {c, rp, 0, 0} and {c, rp, 1, 0}
__global__ void k_bos_pool(BosDev d) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= (int64_t)d.n_rp * d.Q) return;
    const int rp = (int)(i / d.Q), c = (int)(i % d.Q);
    uint64_t w0[4] = {(uint64_t)c, (uint64_t)rp, 0, 0}, w1[4] = {(uint64_t)c, (uint64_t)rp, 1, 0};
    philox4x64_10(w0, d.seed, kPoolKey);
    philox4x64_10(w1, d.seed, kPoolKey);
    const uint64_t w[6] = {w0[0], w0[1], w0[2], w0[3], w1[0], w1[1]};
    float* out = d.pool + i * 6;
#pragma unroll
    for (int a = 0; a < 6; ++a) {
        const int ext = d.box[rp * 12 + (a < 3 ? 3 + a : 6 + 3 + (a - 3))];
        out[a] = __fmul_rn(u24(w[a]), (float)(ext - 1));
    }
}

// Bytes of the propose kernel's first shared region: the pool keys, the two
// 16 KB operand tiles of the shortlist product, or the picks' columns
// (32 x 128 floats), whichever is largest.
__host__ __device__ constexpr size_t propose_region0(int Q) {
    return (size_t)Q * 8 > 32768 ? (size_t)Q * 8 : 32768;
}

// 16-byte global -> shared copy through L2 (cp.async)
__device__ __forceinline__ void bos_cp_async16(void* smem, const void* gmem) {
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(tc::smem_u32(smem)),
                 "l"(gmem)
                 : "memory");
}

// D (TMEM) (+)= A B^T, TF32 operands from shared-memory descriptors
__device__ __forceinline__ void bos_mma_tf32(uint32_t d, uint64_t a, uint64_t b, uint32_t idesc,
                                             uint32_t accum) {
    asm volatile(
        "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n\t}" ::"r"(d),
        "l"(a), "l"(b), "r"(idesc), "r"(accum));
}

// Warp-wide descending sort of 256 unique 64-bit keys, eight per lane in
// blocked order (lane l holds positions 8l .. 8l + 7): a bitonic sorter whose
// stages at distance >= 8 exchange across lanes. An element takes its
// partner's key only when the partner is strictly larger (it keeps the
// maximum) or strictly smaller (it keeps the minimum), so equal keys stay.
__device__ __forceinline__ void warp_sort256_desc(unsigned long long (&k)[8], int lane) {
    const int g0 = lane * 8;
#pragma unroll
    for (int size = 2; size <= 256; size <<= 1) {
#pragma unroll
        for (int d = size >> 1; d > 0; d >>= 1) {
            if (d >= 8) {
                const bool keep_max = ((g0 & d) == 0) == ((g0 & size) == 0);
#pragma unroll
                for (int e = 0; e < 8; ++e) {
                    const unsigned long long o = __shfl_xor_sync(0xffffffffu, k[e], d / 8);
                    k[e] = (keep_max ? o > k[e] : o < k[e]) ? o : k[e];
                }
            } else {
#pragma unroll
                for (int e = 0; e < 8; ++e) {
                    const int e2 = e ^ d;
                    if (e2 > e) {
                        const bool desc = ((g0 + e) & size) == 0;
                        const unsigned long long a = k[e], b = k[e2];
                        const bool swap = desc ? b > a : b < a;
                        k[e] = swap ? b : a;
                        k[e2] = swap ? a : b;
                    }
                }
            }
        }
    }
}

// Descending order of a bitonic sequence of 128 keys, four per lane in
// blocked order: the bitonic merger.
__device__ __forceinline__ void warp_merge128_desc(unsigned long long (&k)[4], int lane) {
    const int g0 = lane * 4;
#pragma unroll
    for (int d = 64; d > 0; d >>= 1) {
        if (d >= 4) {
            const bool keep_max = (g0 & d) == 0;
#pragma unroll
            for (int e = 0; e < 4; ++e) {
                const unsigned long long o = __shfl_xor_sync(0xffffffffu, k[e], d / 4);
                k[e] = (keep_max ? o > k[e] : o < k[e]) ? o : k[e];
            }
        } else {
#pragma unroll
            for (int e = 0; e < 4; ++e) {
                const int e2 = e ^ d;
                if (e2 > e) {
                    const unsigned long long a = k[e], b = k[e2];
                    k[e] = a > b ? a : b;
                    k[e2] = a > b ? b : a;
                }
            }
        }
    }
}

// ---------------------------------------------------------------------------
// propose: one CTA per region pair. Dynamic smem: Q keys (8 B), M shortlist
// ids, M x M covariance, M x 6 positions, M means, a row buffer.
__global__ void __launch_bounds__(kBosThreads) k_bos_propose(BosDev d) {
    extern __shared__ __align__(16) unsigned char bs[];
    const int rp = blockIdx.x, tid = threadIdx.x;
    const int r = *d.round, R = d.R, Q = d.Q, M = d.M;
    unsigned* sel = d.sel + (int64_t)rp * (Q / 32);
    int* picks = d.picks + rp * R;
    if (r == 0) {
        if (tid < R) {
            picks[tid] = tid;
            atomicOr(&sel[tid >> 5], 1u << (tid & 31));
        }
        return;
    }
    const int s = obs_before(r, R, d.L), L = d.L;
    if (tid < L) picks[tid] = -1;  // local proposals: positions made by k_bos_round_pairs
    // shared memory: region0 (1024-byte aligned) holds the pool keys, then the
    // product's operand tiles, then the picks' columns
    unsigned char* region0 = reinterpret_cast<unsigned char*>(
        (reinterpret_cast<uintptr_t>(bs) + 1023) & ~uintptr_t(1023));
    unsigned long long* key = reinterpret_cast<unsigned long long*>(region0);
    int* SL = reinterpret_cast<int*>(region0 + propose_region0(Q));
    float* cov = reinterpret_cast<float*>(SL + M);
    float* pos = cov + M * M;
    float* msl = pos + M * 6;
    float* red_v = msl + M;  // 32 scalars
    uint64_t* bar = reinterpret_cast<uint64_t*>(red_v + 32);  // 2 mbarriers
    uint32_t* tslot = reinterpret_cast<uint32_t*>(bar + 2);
    volatile int* abort_flag = reinterpret_cast<volatile int*>(tslot + 1);
    const float* mu = d.mu + (int64_t)rp * Q;
    const float* var = d.var + (int64_t)rp * Q;
    const float kappa = d.kappa, sf2 = d.hyp[rp * 4 + 1], sn2 = d.hyp[rp * 4 + 2];
    for (int c = tid; c < Q; c += blockDim.x) {
        const bool taken = (sel[c >> 5] >> (c & 31)) & 1u;
        const float u = mu[c] + kappa * sqrtf(fmaxf(var[c], 0.f));
        key[c] = taken ? 0ull
                       : ((unsigned long long)okey32(u) << 32) | (0xffffffffull - (unsigned)c);
    }
    __syncthreads();
    // the M largest keys, in descending order: each warp sorts 256-key
    // segments of the pool in registers (eight keys per lane) and keeps each
    // segment's top 128 in place; a tree of pairwise merges (the top 128 of
    // two descending lists: the elementwise maximum against the other list
    // reversed is bitonic and holds them, a bitonic merger orders it) leaves
    // the 128 largest in segment 0. Keys are unique apart from the zero keys
    // of taken entries, so the shortlist and its order are those of a full
    // descending sort.
    {
        const int warp = tid >> 5, lane = tid & 31, nseg = Q / 256;
        for (int sg = warp; sg < nseg; sg += kBosThreads / 32) {
            unsigned long long k8[8];
#pragma unroll
            for (int e = 0; e < 8; ++e) k8[e] = key[sg * 256 + lane * 8 + e];
            warp_sort256_desc(k8, lane);
            if (lane < 16) {
#pragma unroll
                for (int e = 0; e < 8; ++e) key[sg * 256 + lane * 8 + e] = k8[e];
            }
        }
        __syncthreads();
        for (int w = 1; w < nseg; w <<= 1) {
            for (int m = warp; m * 2 * w < nseg; m += kBosThreads / 32) {
                const int sa = m * 2 * w * 256, sb = sa + w * 256;
                unsigned long long k4[4];
#pragma unroll
                for (int e = 0; e < 4; ++e) {
                    const unsigned long long a = key[sa + lane * 4 + e],
                                             b = key[sb + 127 - lane * 4 - e];
                    k4[e] = a > b ? a : b;
                }
                warp_merge128_desc(k4, lane);
#pragma unroll
                for (int e = 0; e < 4; ++e) key[sa + lane * 4 + e] = k4[e];
            }
            __syncthreads();
        }
    }
    float inv_ell[6];
    inv_ell_of(d, rp, inv_ell);
    for (int i = tid; i < M; i += blockDim.x) {
        const int c = (int)(0xffffffffull - (key[i] & 0xffffffffull));
        SL[i] = c;
        msl[i] = mu[c];
#pragma unroll
        for (int a = 0; a < 6; ++a) pos[i * 6 + a] = d.pool[((int64_t)rp * Q + c) * 6 + a];
    }
    __syncthreads();
    // posterior covariance among the shortlist: K(SL, SL) - X^T X with
    // X = V[:, SL] (s observations x M entries), on the tensor cores: per
    // K step three TF32 products X_hi X_hi + X_hi X_lo + X_lo X_hi, where
    // X_hi keeps the first 11 significant bits of X and X_lo = X - X_hi
    // exactly (the dropped X_lo X_lo term and the 11-bit reading of X_lo are
    // below 2^-20 relative), FP32 accumulation in TMEM. The operand tiles
    // are 128 rows (entries, zero beyond M) x 32 observations, K-major with
    // the 128-byte swizzle; A and B are the same tiles. One stage: the next
    // block's loads are issued while the MMAs of the current one run.
    const int Sp = d.Sp;
    const float* Vr = d.V + (int64_t)rp * Q * Sp;  // pool-major columns of Sp rows
    const int warp = tid >> 5, lane = tid & 31;
    unsigned char* Xh = region0;
    unsigned char* Xl = region0 + 128 * 128;
    if (tid == 0) {
        tc::mbar_init(&bar[0], 1);
        tc::mbar_init(&bar[1], 1);
        *abort_flag = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                         tc::smem_u32(tslot)),
                     "r"(128));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
    }
    tc::tc_fence_before();
    __syncthreads();
    tc::tc_fence_after();
    const uint32_t tmem = *tslot;
    const int srow = tid >> 1, sc0 = (tid & 1) * 4;  // staging unit: row, four 16-byte chunks
    const float* src = Vr + (int64_t)(srow < M ? SL[srow] : 0) * Sp;
    float4 nx[4];
    auto load_blk = [&](int t0) {
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            const int t = t0 + 4 * (sc0 + q);  // rows at and beyond s read as zero in V
            nx[q] = (srow < M && t < s) ? __ldcs(reinterpret_cast<const float4*>(src + t))
                                        : make_float4(0.f, 0.f, 0.f, 0.f);
        }
    };
    auto split = [](float x, float& hi) {
        hi = __uint_as_float(__float_as_uint(x) & 0xffffe000u);
        return x - hi;
    };
    const int nkb = (s + 31) / 32;
    const uint32_t idesc = (1u << 4) | (2u << 7) | (2u << 10) | ((uint32_t)(M >> 3) << 17) |
                           ((uint32_t)(128 >> 4) << 24);  // FP32 += TF32 x TF32, K-major
    load_blk(0);
    for (int kb = 0; kb < nkb; ++kb) {
        if (kb > 0 && !*abort_flag && !tc::mbar_wait(&bar[0], (kb - 1) & 1, abort_flag)) {
            *abort_flag = 1;
            set_status(d.status, DEV_TIMEOUT);
        }
        __syncthreads();  // the previous block's MMAs have read the tiles
        if (*abort_flag) break;
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            float4 h, l;
            l.x = split(nx[q].x, h.x);
            l.y = split(nx[q].y, h.y);
            l.z = split(nx[q].z, h.z);
            l.w = split(nx[q].w, h.w);
            const uint32_t off = (uint32_t)(srow * 128 + (((sc0 + q) ^ (srow & 7)) << 4));
            *reinterpret_cast<float4*>(Xh + off) = h;
            *reinterpret_cast<float4*>(Xl + off) = l;
        }
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        __syncthreads();
        if (tid == 0) {
            tc::tc_fence_after();
            const uint32_t bh = tc::smem_u32(Xh), bl = tc::smem_u32(Xl);
#pragma unroll
            for (int k = 0; k < 4; ++k) {
                const uint64_t dh = tc::sdesc(bh + k * 32), dl = tc::sdesc(bl + k * 32);
                bos_mma_tf32(tmem, dh, dh, idesc, (kb | k) != 0);
                bos_mma_tf32(tmem, dh, dl, idesc, 1);
                bos_mma_tf32(tmem, dl, dh, idesc, 1);
            }
            tc::mma_commit(&bar[0]);
        }
        if (kb + 1 < nkb) load_blk(32 * (kb + 1));
    }
    if (!*abort_flag && !tc::mbar_wait(&bar[0], (nkb - 1) & 1, abort_flag)) {
        *abort_flag = 1;
        set_status(d.status, DEV_TIMEOUT);
    }
    __syncthreads();
    const bool ok = !*abort_flag;
    if (ok) {
        // warp w reads TMEM lanes 32 (w % 4) .. + 31 (rows) and 64 columns;
        // column c of the covariance goes to cov[c M + row] (lanes write
        // consecutive words), so row c of cov is column c
        tc::tc_fence_after();
        const int row = 32 * (warp & 3) + lane, cb = 64 * (warp >> 2);
        const uint32_t taddr = tmem + ((uint32_t)(32 * (warp & 3)) << 16) + (uint32_t)cb;
#pragma unroll 1
        for (int h = 0; h < 2; ++h) {
            float v[32];
            tc::tmem_ld32(taddr + 32 * h, v);
#pragma unroll
            for (int i = 0; i < 32; ++i) {
                const int col = cb + 32 * h + i;
                if (row < M && col < M)
                    cov[col * M + row] = matern52(pos + row * 6, pos + col * 6, inv_ell, sf2) - v[i];
            }
        }
    } else if (tid == 0) {  // every issued MMA completes before TMEM is released
        tc::mma_commit(&bar[1]);
        tc::mbar_wait(&bar[1], 0, nullptr);
    }
    tc::tc_fence_before();
    __syncthreads();
    if (warp == 0) {
        tc::tc_fence_after();
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(128));
    }
    if (!ok) return;
    // greedy picks with the kriging-believer update (the R - L pool
    // proposals), by warp 0 alone. The UCB needs only the diagonal of the
    // updated covariance, and the column of pick j is cov0[:, c_j] minus the
    // terms of the earlier picks, col_p col_p[c_j] / (col_p[c_p] + noise): the
    // same operations in the same order as subtracting every rank-one update
    // from the whole matrix, on j + 1 columns instead of M. cov0 is exactly
    // symmetric (both triangles are the same products), so column c is read
    // as row c.
    if (tid >= 32) return;
    float* colbuf = reinterpret_cast<float*>(region0);  // [R - L][M]: the picks' columns
    float* invb = red_v;     // [R - L]: 1 / (col_p[c_p] + noise)
    float dg[4];
    bool tk[4];
#pragma unroll
    for (int q = 0; q < 4; ++q) {
        const int i = lane + 32 * q;
        dg[q] = i < M ? cov[i * M + i] : 0.f;
        tk[q] = i >= M;
    }
    for (int j = 0; j < R - L; ++j) {
        float bv = -CUDART_INF_F;
        int bi = 0x7fffffff;
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            const int i = lane + 32 * q;
            if (tk[q]) continue;
            const float u = msl[i] + kappa * sqrtf(fmaxf(dg[q], 0.f));
            if (u > bv || (u == bv && i < bi)) {
                bv = u;
                bi = i;
            }
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            const float ov = __shfl_xor_sync(0xffffffffu, bv, o);
            const int oi = __shfl_xor_sync(0xffffffffu, bi, o);
            if (ov > bv || (ov == bv && oi < bi)) {
                bv = ov;
                bi = oi;
            }
        }
        const int c = bi;
        if (lane == 0) {
            picks[L + j] = SL[c];
            atomicOr(&sel[SL[c] >> 5], 1u << (SL[c] & 31));
        }
        float x[4], xc = 0.f;
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            const int i = lane + 32 * q;
            float v = i < M ? cov[c * M + i] : 0.f;
            for (int p = 0; p < j; ++p) v -= colbuf[p * M + i] * colbuf[p * M + c] * invb[p];
            x[q] = v;
            if (q == (c >> 5)) xc = v;
        }
        xc = __shfl_sync(0xffffffffu, xc, c & 31);
        const float inv = 1.f / (xc + sn2);
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            const int i = lane + 32 * q;
            if (i < M) colbuf[j * M + i] = x[q];
            dg[q] -= x[q] * x[q] * inv;
            tk[q] = tk[q] || i == c;
        }
        if (lane == 0) invb[j] = inv;
        __syncwarp();
    }
}

// ---------------------------------------------------------------------------
// probabilistic reparameterization of proposal j: blocks {j, rp, 2 + r, 0/1}.
// A local proposal (pick -1) first gets its position from incumbent j mod 2
// (the only one when a single sample exists): theta_d = clip(theta_inc,d +
// lscale ext_d z_d, 0, ext_d - 1) with six Box-Muller normals from blocks
// {j, rp, 2 + r, 2/3}: for i = 0..2, u1 = (top 24 bits of w[2i] + 1) 2^-24,
// u2 = top 24 bits of w[2i+1] 2^-24, z = sqrt(-2 ln u1) (cos, sin)(2 pi u2).
__global__ void k_bos_round_pairs(BosDev d) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= d.n_rp * d.R) return;
    const int rp = i / d.R, j = i % d.R, r = *d.round;
    const int c = d.picks[rp * d.R + j];
    const int* bx = d.box + rp * 12;
    float th[6];
    if (c >= 0) {
#pragma unroll
        for (int a = 0; a < 6; ++a) th[a] = d.pool[((int64_t)rp * d.Q + c) * 6 + a];
    } else {
        const int ninc = min(2, r * d.R);
        const int src = max(d.inc_idx[rp * 2 + j % ninc], 0);  // set after every round
        const float* ti = d.theta + ((int64_t)rp * d.R * d.T + src) * 6;
        uint64_t w0[4] = {(uint64_t)j, (uint64_t)rp, (uint64_t)(2 + r), 2};
        uint64_t w1[4] = {(uint64_t)j, (uint64_t)rp, (uint64_t)(2 + r), 3};
        philox4x64_10(w0, d.seed, kRoundKey);
        philox4x64_10(w1, d.seed, kRoundKey);
        const uint64_t w[8] = {w0[0], w0[1], w0[2], w0[3], w1[0], w1[1], w1[2], w1[3]};
#pragma unroll
        for (int q = 0; q < 3; ++q) {
            const float u1 = (float)((w[2 * q] >> 40) + 1) * 5.9604644775390625e-8f;  // 2^-24
            const float u2 = (float)(w[2 * q + 1] >> 40) * 5.9604644775390625e-8f;
            const float rad = sqrtf(-2.f * logf(u1));
            float sn, cs;
            sincospif(2.f * u2, &sn, &cs);
#pragma unroll
            for (int h = 0; h < 2; ++h) {
                const int a = 2 * q + h;
                const int ext = bx[a < 3 ? 3 + a : 6 + 3 + (a - 3)];
                const float z = h ? rad * sn : rad * cs;
                th[a] = fminf(fmaxf(fmaf(d.lscale * (float)ext, z, ti[a]), 0.f), (float)(ext - 1));
            }
        }
    }
    float* hist = d.theta + ((int64_t)rp * d.R * d.T + (int64_t)r * d.R + j) * 6;
#pragma unroll
    for (int a = 0; a < 6; ++a) hist[a] = th[a];
    uint64_t w0[4] = {(uint64_t)j, (uint64_t)rp, (uint64_t)(2 + r), 0};
    uint64_t w1[4] = {(uint64_t)j, (uint64_t)rp, (uint64_t)(2 + r), 1};
    philox4x64_10(w0, d.seed, kRoundKey);
    philox4x64_10(w1, d.seed, kRoundKey);
    const uint64_t w[6] = {w0[0], w0[1], w0[2], w0[3], w1[0], w1[1]};
    int v[6];
#pragma unroll
    for (int a = 0; a < 6; ++a) {
        const float f = floorf(th[a]);
        v[a] = (int)f + (u24(w[a]) < __fsub_rn(th[a], f) ? 1 : 0);
    }
    if (d.self[rp]) {  // a self pair never pairs a point with itself
        if (v[0] == v[3] && v[1] == v[4] && v[2] == v[5]) {
            const int np = bx[3] * bx[4] * bx[5];
            int l = v[3] + bx[3] * (v[4] + bx[4] * v[5]);
            l = (l + 1) % np;
            v[3] = l % bx[3];
            v[4] = (l / bx[3]) % bx[4];
            v[5] = l / (bx[3] * bx[4]);
        }
    }
    d.pa[i] = (uint32_t)((bx[0] + v[0]) + d.X * ((bx[1] + v[1]) + d.Y * (bx[2] + v[2])));
    d.pb[i] = (uint32_t)((bx[6] + v[3]) + d.X * ((bx[7] + v[4]) + d.Y * (bx[8] + v[5])));
}

// ---------------------------------------------------------------------------
// KSG candidates of the evaluation are walked as a sample stream (two staging
// slots per warp) for 32 <= n <= 256, one candidate per warp otherwise
__host__ __device__ __forceinline__ bool eval_stream(int n, int n_pad) {
    return n >= 32 && n_pad <= 256;
}

// evaluate: persistent work queue over (measure, pair) items, KSG first.
template <int KMAX>
__global__ void k_bos_eval(BosDev d, int warps_per_block) {
    extern __shared__ __align__(16) unsigned char es[];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int n = d.n, n_pad = d.n_pad, B = d.bins;
    long long* psi = reinterpret_cast<long long*>(es);
    long long* clogc = psi + ((n + 2) & ~1);
    const size_t slot = ksg_slot_bytes(n_pad, KMAX);
    const bool stream = eval_stream(n, n_pad);
    const int slots = stream ? 2 : 1;
    unsigned char* wbase = reinterpret_cast<unsigned char*>(clogc + ((n + 2) & ~1)) +
                           (size_t)warp * (slots * slot + 256 * sizeof(int));
    int* hist = reinterpret_cast<int*>(wbase + slots * slot);
    for (int i = threadIdx.x; i <= n; i += blockDim.x) {
        psi[i] = d.psi_fix[i];
        clogc[i] = d.clogc_fix[i];
    }
    for (int c = lane; c < B * B; c += 32) hist[c] = 0;
    __syncthreads();
    const int per = d.n_rp * d.R, total = 4 * per;
    // KSG first (the longest measure): for 32 <= n <= 256 a warp takes chunks of
    // kEvalChunk consecutive candidates and walks their samples as one
    // stream, 32 per round, with two staging slots (a round spans at most two
    // candidates; a candidate's slot is restaged for the one two places
    // later, whose first sample lies beyond the round that ends it)
    if (stream) {
        while (true) {
            int c0 = 0;
            if (lane == 0) c0 = atomicAdd(d.queue + 1, kEvalChunk);
            c0 = __shfl_sync(0xffffffffu, c0, 0);
            if (c0 >= per) break;
            const int c1 = min(per, c0 + kEvalChunk);
            int tr = c0, tir = 0, staged = c0;
            long long acc[2] = {0, 0};
            while (tr < c1) {
                const int t_last = min(c1 - 1, tr + (tir + 31 >= n ? 1 : 0));
                for (; staged <= t_last; ++staged) {  // warp-uniform
                    const int64_t ra = (int64_t)d.pa[staged] * n_pad,
                                  rb = (int64_t)d.pb[staged] * n_pad;
                    ksg_stage<KMAX>(wbase + (staged & 1) * slot, n, n_pad, d.sorted + ra,
                                    d.perm + ra, d.fvals + ra, d.sorted_b + rb, d.perm_b + rb,
                                    d.fvals_b + rb);
                }
                int ti = tir + lane, tt = tr;
                if (ti >= n) {
                    ti -= n;
                    ++tt;
                }
                if (tt < c1) {
                    const long long v = ksg_sample<KMAX>(wbase + (tt & 1) * slot, n, n_pad, d.k,
                                                         ti, psi, nullptr, nullptr, nullptr);
                    if (tt & 1) acc[1] += v;
                    else acc[0] += v;
                }
                if (tir + 32 >= n) {  // candidate tr ends in this round
                    const long long sum = warp_sum_i64((tr & 1) ? acc[1] : acc[0]);
                    if (lane == 0)
                        d.vals[(int64_t)CC_MI_KSG * per + tr] =
                            (float)(d.psi_nk - (double)sum * d.fix_over_n);
                    if (tr & 1) acc[1] = 0;
                    else acc[0] = 0;
                }
                __syncwarp();
                tir += 32;
                if (tir >= n) {
                    tir -= n;
                    ++tr;
                }
            }
        }
    }
    const int first = stream ? per : 0;  // the items left to the queue below
    while (true) {
        int item = 0;
        if (lane == 0) item = first + atomicAdd(d.queue, 1);
        item = __shfl_sync(0xffffffffu, item, 0);
        if (item >= total) break;
        const int measure = 3 - item / per, t = item % per;
        const uint32_t p = d.pa[t], q = d.pb[t];
        const int64_t ra = (int64_t)p * n_pad, rb = (int64_t)q * n_pad;
        float value = 0.f;
        if (measure == CC_MI_KSG) {
            ksg_stage<KMAX>(wbase, n, n_pad, d.sorted + ra, d.perm + ra, d.fvals + ra,
                            d.sorted_b + rb, d.perm_b + rb, d.fvals_b + rb);
            long long acc = 0;
            for (int ti = lane; ti < n; ti += 32)
                acc += ksg_sample<KMAX>(wbase, n, n_pad, d.k, ti, psi, nullptr, nullptr, nullptr);
            acc = warp_sum_i64(acc);
            value = (float)(d.psi_nk - (double)acc * d.fix_over_n);
        } else if (measure == CC_MI_BINNED) {
            const uint8_t* ba = d.bins_p + ra;
            const uint8_t* bb = d.bins_b + rb;
            // the member whose increment finds its cell empty owns the cell:
            // it adds the cell's c ln c once the counts are complete and clears it
            unsigned own = 0;  // bit j: member lane + 32 j (n <= 1024)
            for (int m = lane, j = 0; m < n; m += 32, ++j)
                if (atomicAdd(&hist[ba[m] * B + bb[m]], 1) == 0) own |= 1u << j;
            __syncwarp();
            long long s = 0;
            for (unsigned o = own; o; o &= o - 1) {
                const int m = lane + 32 * (__ffs(o) - 1);
                s += clogc[hist[ba[m] * B + bb[m]]];
            }
            __syncwarp();
            for (unsigned o = own; o; o &= o - 1) {
                const int m = lane + 32 * (__ffs(o) - 1);
                hist[ba[m] * B + bb[m]] = 0;
            }
            s = warp_sum_i64(s);
            value = (float)(d.logn + (double)(s - d.hmarg[p] - d.hmarg_b[q]) * d.fix_over_n);
        } else {
            const float* A = (measure == CC_SPEARMAN ? d.rhat : d.zhat) + ra;
            const float* Bp = (measure == CC_SPEARMAN ? d.rhat_b : d.zhat_b) + rb;
            float acc = 0.f;
            for (int m = lane; m < n_pad; m += 32) acc = fmaf(A[m], Bp[m], acc);
            value = warp_sum_f32(acc);
        }
        if (lane == 0) d.vals[(int64_t)measure * per + t] = value;
        __syncwarp();
    }
}

// running extremes per (measure, region pair); index = (pa << 32) | pb
__global__ void k_bos_extremes(BosDev d) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= 4 * d.n_rp) return;
    const int m = i / d.n_rp, rp = i % d.n_rp, per = d.n_rp * d.R;
    Partial b = d.best[i];
    if (*d.round == 0) {
        b.max = -CUDART_INF_F;
        b.min = CUDART_INF_F;
        b.argmax = b.argmin = ~0ull;
        b.count = 0;
    }
    for (int j = 0; j < d.R; ++j) {
        const int t = rp * d.R + j;
        const float v = d.vals[(int64_t)m * per + t];
        const unsigned long long id = ((unsigned long long)d.pa[t] << 32) | d.pb[t];
        if (v > b.max || (v == b.max && id < b.argmax)) {
            b.max = v;
            b.argmax = id;
        }
        if (v < b.min || (v == b.min && id < b.argmin)) {
            b.min = v;
            b.argmin = id;
        }
        b.count++;
    }
    d.best[i] = b;
    if (m == d.objective) {
        // the objective's value of every sample, and the two best so far (the
        // earlier sample on ties: strictly greater values replace)
        const int r = *d.round;
        float v0 = r ? d.inc_val[rp * 2] : -CUDART_INF_F;
        float v1 = r ? d.inc_val[rp * 2 + 1] : -CUDART_INF_F;
        int i0 = r ? d.inc_idx[rp * 2] : -1, i1 = r ? d.inc_idx[rp * 2 + 1] : -1;
        for (int j = 0; j < d.R; ++j) {
            const float v = d.vals[(int64_t)m * per + rp * d.R + j];
            const int idx = r * d.R + j;
            d.yall[(int64_t)rp * d.R * d.T + idx] = v;
            if (v > v0) {
                v1 = v0;
                i1 = i0;
                v0 = v;
                i0 = idx;
            } else if (v > v1) {
                v1 = v;
                i1 = idx;
            }
        }
        d.inc_val[rp * 2] = v0;
        d.inc_val[rp * 2 + 1] = v1;
        d.inc_idx[rp * 2] = i0;
        d.inc_idx[rp * 2 + 1] = i1;
    }
}

// ---------------------------------------------------------------------------
// condition: one CTA per region pair absorbs the round's R observations.
__global__ void __launch_bounds__(kBosThreads) k_bos_condition(BosDev d) {
    extern __shared__ __align__(16) unsigned char cs[];
    const int rp = blockIdx.x, tid = threadIdx.x, lane = tid & 31;
    const int r = *d.round, R = d.R, Q = d.Q, S = d.S;
    // the round's GP observations: all R proposals in round 0, the R - L pool
    // proposals (after the local ones) later; nn <= R, matrices use stride nn
    const int s = obs_before(r, R, d.L), nn = obs_new(r, R, d.L), j0 = r == 0 ? 0 : d.L;
    // G (kGRows x 32 of V[:, P], 0-padded) is 1024-byte aligned: the operand
    // tiles of the product below reuse its space
    unsigned char* cs_al = reinterpret_cast<unsigned char*>(
        (reinterpret_cast<uintptr_t>(cs) + 1023) & ~uintptr_t(1023));
    float* G = reinterpret_cast<float*>(cs_al);
    double* Lf = reinterpret_cast<double*>(cs_al + kCondRegion0);  // R x R (fp64 Cholesky)
    float* covP = reinterpret_cast<float*>(Lf + R * R);    // R x R
    float* L = covP + R * R;                               // R x R fp32 copy
    float* gb = L + R * R;                        // R: V[:, P]^T beta
    float* b2 = gb + R;                           // R: new beta
    float* pp = b2 + R;                           // R x 6 pick positions
    float* yv = pp + R * 6;                       // R
    float* mP = yv + R;                           // R prior at picks
    float* hyp = mP + R;                          // 4
    float* Linv = hyp + 4;                        // R: 1 / L22[i][i]
    uint64_t* cbar = reinterpret_cast<uint64_t*>(Linv + R + (R & 1));  // 6 mbarriers
    uint32_t* tslot = reinterpret_cast<uint32_t*>(cbar + 6);
    volatile int* abort_flag = reinterpret_cast<volatile int*>(tslot + 1);
    const int* P = d.picks + rp * R + j0;
    const int per = d.n_rp * R;
    const int Sp = d.Sp;
    float* Vr = d.V + (int64_t)rp * Q * Sp;  // pool-major columns of Sp rows
    float* mu = d.mu + (int64_t)rp * Q;
    float* var = d.var + (int64_t)rp * Q;
    if (tid < nn) {
        yv[tid] = d.vals[(int64_t)d.objective * per + rp * R + j0 + tid];
#pragma unroll
        for (int a = 0; a < 6; ++a) pp[tid * 6 + a] = d.pool[((int64_t)rp * Q + P[tid]) * 6 + a];
    }
    __syncthreads();
    if (r == 0 && tid == 0) {
        float m = 0.f, v = 0.f;
        for (int j = 0; j < R; ++j) m += yv[j];
        m /= R;
        for (int j = 0; j < R; ++j) v += (yv[j] - m) * (yv[j] - m);
        v = fmaxf(v / R, 1e-12f);
        d.hyp[rp * 4 + 0] = m;
        d.hyp[rp * 4 + 1] = v;
        d.hyp[rp * 4 + 2] = 1e-4f * v;
    }
    __syncthreads();
    if (tid < 4) hyp[tid] = d.hyp[rp * 4 + tid];
    __syncthreads();
    const float m0 = hyp[0], sf2 = hyp[1], sn2 = hyp[2];
    if (r == 0) {
        for (int c = tid; c < Q; c += blockDim.x) {
            mu[c] = d.prior ? d.prior[(int64_t)rp * Q + c] : m0;
            var[c] = sf2;
        }
    }
    if (tid < nn) mP[tid] = d.prior ? d.prior[(int64_t)rp * Q + P[tid]] : m0;
    float inv_ell[6];
    inv_ell_of(d, rp, inv_ell);
    // covP = V[:, P]^T V[:, P] and gb = V[:, P]^T beta over the s old rows.
    // G holds up to kGRows rows of V[:, P] at a time (most rounds: all of them)
    float cacc[4] = {0.f, 0.f, 0.f, 0.f};  // entries tid, tid+256, ... of R x R
    float gacc = 0.f;
    // G[t][j] = V[t0 + t][P[j]] for t < rows rounded up to 8, zero beyond s and nn
    auto gather = [&](int t0, int rows) {
        const int rp8 = (rows + 7) & ~7;
        for (int e = tid; e < rp8 * 32; e += blockDim.x) {
            const int t = t0 + (e >> 5), j = e & 31;
            G[e] = (t < s && j < nn) ? Vr[(int64_t)P[j] * Sp + t] : 0.f;
        }
    };
    for (int t0 = 0; t0 < s; t0 += kGRows) {
        const int rows = min(kGRows, s - t0);
        __syncthreads();
        gather(t0, rows);
        __syncthreads();
        for (int q = 0; q < 4; ++q) {
            const int e = tid + q * blockDim.x;
            if (e < nn * nn) {
                const int i = e / nn, j = e % nn;
                float a = cacc[q];
                for (int t = 0; t < rows; ++t) a = fmaf(G[t * 32 + i], G[t * 32 + j], a);
                cacc[q] = a;
            }
        }
        if (tid < nn)
            for (int t = 0; t < rows; ++t)
                gacc = fmaf(G[t * 32 + tid], d.beta[(int64_t)rp * S + t0 + t], gacc);
    }
    for (int q = 0; q < 4; ++q) {
        const int e = tid + q * blockDim.x;
        if (e < nn * nn) {
            const int i = e / nn, j = e % nn;
            covP[e] = matern52(pp + i * 6, pp + j * 6, inv_ell, sf2) - cacc[q] + (i == j ? sn2 : 0.f);
        }
    }
    if (tid < nn) gb[tid] = gacc;
    __syncthreads();
    // Cholesky of covP (fp64, warp 0, lane i owns row i), right-looking: at
    // step j the pivot's reciprocal square root scales column j and the
    // trailing rows subtract their column-j products, so each entry sees
    // the same subtractions in the same order as the column-by-column form
    // while all rows work at once (this GPU's FP64 pipe is narrow).
    if (tid < 32) {
        for (int e = lane; e < nn * nn; e += 32) Lf[e] = (double)covP[e];
        __syncwarp();
        for (int j = 0; j < nn; ++j) {
            const double x = fmax(Lf[j * nn + j], 1e-12 * (double)sf2);
            const double rj = rsqrt(x);
            const bool below = lane > j && lane < nn;
            const double lij = below ? Lf[lane * nn + j] * rj : 0.0;
            __syncwarp();  // column j is read before it is overwritten
            if (lane == j) {
                Lf[j * nn + j] = x * rj;
                Linv[j] = (float)rj;
            } else if (below) {
                Lf[lane * nn + j] = lij;
            }
            __syncwarp();
            if (below)
                for (int q = j + 1; q <= lane; ++q) Lf[lane * nn + q] -= lij * Lf[q * nn + j];
            __syncwarp();
        }
        for (int e = lane; e < nn * nn; e += 32) {
            const int i = e / nn, j = e % nn;
            L[e] = j <= i ? (float)Lf[e] : 0.f;
        }
        // beta2 = L22^-1 (y - m_P - V[:, P]^T beta1), forward substitution
        // by columns: lane q keeps its right-hand side
        double v = lane < nn ? (double)yv[lane] - mP[lane] - gb[lane] : 0.0;
        for (int i = 0; i < nn; ++i) {
            const double vi = __shfl_sync(0xffffffffu, v, i);
            const float bi = (float)(vi / Lf[i * nn + i]);
            if (lane == i) b2[i] = bi;
            if (lane > i && lane < nn) v -= Lf[lane * nn + i] * (double)bi;
        }
    }
    __syncthreads();
    // new rows: V2 = L22^-1 (K(P, pool) - W) with W = V[:, P]^T V, then the
    // mean and variance updates of every pool entry (finish below).
    auto finish = [&](int c, float (&w)[32]) {
        const float* pc = d.pool + ((int64_t)rp * Q + c) * 6;
        float pcl[6];
#pragma unroll
        for (int a = 0; a < 6; ++a) pcl[a] = pc[a];
        float dv = 0.f, dm = 0.f;
#pragma unroll
        for (int i = 0; i < 32; ++i) {
            if (i < nn) {
                float x = matern52(pp + i * 6, pcl, inv_ell, sf2) - w[i];
#pragma unroll
                for (int q = 0; q < i; ++q) x = fmaf(-L[i * nn + q], w[q], x);
                x *= Linv[i];
                w[i] = x;
                Vr[(int64_t)c * Sp + s + i] = x;
                dv = fmaf(x, x, dv);
                dm = fmaf(x, b2[i], dm);
            }
        }
        var[c] -= dv;
        mu[c] += dm;
    };
    if (s == 0) {  // round 0: no earlier observations, W = 0
        for (int c = tid; c < Q; c += blockDim.x) {
            float w[32];
#pragma unroll
            for (int i = 0; i < 32; ++i) w[i] = 0.f;
            finish(c, w);
        }
    } else {
        // W^T (Q x 32) = V^T G on the tensor cores, per tile of 128 pool
        // entries (the MMA's M) and the picks padded to 32 (N), K = the s
        // observations in blocks of 32: three TF32 products per K step
        // (hi x hi + hi x lo + lo x hi, x = hi + lo with hi the first 11
        // significant bits), FP32 accumulation in TMEM. Warps 4-7 stage the
        // operand tiles (K-major, 128-byte swizzle, one stage; the next
        // block's loads are in flight while the MMAs run) and lane 0 of warp
        // 4 issues the MMAs into one of two TMEM accumulators; warps 0-3 read
        // a finished tile's accumulator (TMEM lane = pool entry) and run its
        // entries' finish while the next tile is multiplied. Every wait is
        // bounded; on timeout the block records DEV_TIMEOUT, the roles leave
        // their loops, issued MMAs are drained and TMEM is freed.
        unsigned char* Ah = cs_al;         // 128 x 128 B
        unsigned char* Al = Ah + 16384;
        unsigned char* Bh = Al + 16384;    // 32 x 128 B
        unsigned char* Bl = Bh + 4096;
        uint64_t* sfree = &cbar[0];   // the stage's MMAs have completed
        uint64_t* afull = &cbar[1];   // [2] accumulator b holds a finished tile
        uint64_t* aempty = &cbar[3];  // [2] accumulator b has been read
        uint64_t* drain = &cbar[5];
        const int warp = tid >> 5, ntile = Q / 128, nkb = (s + 31) / 32;
        __syncthreads();  // G is no longer read: its space becomes the stage
        if (tid == 0) {
            tc::mbar_init(sfree, 1);
            tc::mbar_init(&afull[0], 1);
            tc::mbar_init(&afull[1], 1);
            tc::mbar_init(&aempty[0], 4);
            tc::mbar_init(&aempty[1], 4);
            tc::mbar_init(drain, 1);
            *abort_flag = 0;
            asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        }
        if (warp == 0) {
            asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                             tc::smem_u32(tslot)),
                         "r"(64));
            asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
        }
        tc::tc_fence_before();
        __syncthreads();
        tc::tc_fence_after();
        const uint32_t tmem = *tslot;
        auto fail = [&]() {
            *abort_flag = 1;
            set_status(d.status, DEV_TIMEOUT);
        };
        if (warp >= 4) {  // producers
            const int pt = tid - 128;
            const uint32_t idesc = (1u << 4) | (2u << 7) | (2u << 10) | ((uint32_t)(32 >> 3) << 17) |
                                   ((uint32_t)(128 >> 4) << 24);  // FP32 += TF32 x TF32, K-major
            // block it = (m, kb): A unit q: row (pt + 128 q) >> 3 of tile m, chunk
            // & 7; B unit q: pick (pt + 128 q) >> 3, chunk & 7; rows >= s read as 0.
            // Each producer copies its own ten 16-byte units of a block into a
            // two-block ring (cp.async, [slot][unit][thread]) two blocks ahead
            // of the one it converts, and converts only its own units, so the
            // ring needs no barrier.
            float4* ring = reinterpret_cast<float4*>(Bl + 4096);  // [2][10][128]
            auto issue = [&](int itn) {
                const int mn = itn / nkb, kbn = itn - mn * nkb;
                if (mn < ntile) {
                    const int t0 = 32 * kbn, sl = itn & 1;
#pragma unroll
                    for (int q = 0; q < 8; ++q) {
                        const int u = pt + 128 * q, t = t0 + 4 * (u & 7);
                        if (t < s)
                            bos_cp_async16(&ring[(sl * 10 + q) * 128 + pt],
                                           Vr + (int64_t)(128 * mn + (u >> 3)) * Sp + t);
                    }
#pragma unroll
                    for (int q = 0; q < 2; ++q) {
                        const int u = pt + 128 * q, j = u >> 3, t = t0 + 4 * (u & 7);
                        if (j < nn && t < s)
                            bos_cp_async16(&ring[(sl * 10 + 8 + q) * 128 + pt],
                                           Vr + (int64_t)P[j] * Sp + t);
                    }
                }
                asm volatile("cp.async.commit_group;" ::: "memory");
            };
            auto unit = [&](int itn, int q) {  // this thread's unit q of block itn
                const int kbn = itn % nkb, u = pt + 128 * (q < 8 ? q : q - 8);
                const int t = 32 * kbn + 4 * (u & 7);
                const bool ok = q < 8 ? t < s : ((u >> 3) < nn && t < s);
                return ok ? ring[((itn & 1) * 10 + q) * 128 + pt] : make_float4(0.f, 0.f, 0.f, 0.f);
            };
            auto put = [&](unsigned char* hi, unsigned char* lo, int u, float4 v) {
                float4 h, l;
                h.x = __uint_as_float(__float_as_uint(v.x) & 0xffffe000u);
                h.y = __uint_as_float(__float_as_uint(v.y) & 0xffffe000u);
                h.z = __uint_as_float(__float_as_uint(v.z) & 0xffffe000u);
                h.w = __uint_as_float(__float_as_uint(v.w) & 0xffffe000u);
                l.x = v.x - h.x;
                l.y = v.y - h.y;
                l.z = v.z - h.z;
                l.w = v.w - h.w;
                const int row = u >> 3, ch = u & 7;
                const uint32_t off = (uint32_t)(row * 128 + ((ch ^ (row & 7)) << 4));
                *reinterpret_cast<float4*>(hi + off) = h;
                *reinterpret_cast<float4*>(lo + off) = l;
            };
            auto pbar = []() { asm volatile("bar.sync 1, 128;" ::: "memory"); };
            issue(0);
            issue(1);
            int it = 0;
            for (int m = 0; m < ntile; ++m) {
                for (int kb = 0; kb < nkb; ++kb, ++it) {
                    asm volatile("cp.async.wait_group 1;" ::: "memory");  // block it has landed
                    if (pt == 0 && it > 0 && !*abort_flag &&
                        !tc::mbar_wait(sfree, (it - 1) & 1, abort_flag))
                        fail();
                    pbar();  // the stage is free (or the block gave up)
                    if (*abort_flag) break;
#pragma unroll
                    for (int q = 0; q < 8; ++q) put(Ah, Al, pt + 128 * q, unit(it, q));
#pragma unroll
                    for (int q = 0; q < 2; ++q) put(Bh, Bl, pt + 128 * q, unit(it, 8 + q));
                    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
                    pbar();  // the stage is written
                    if (pt == 0) {
                        const int b = m & 1;
                        if (kb == 0 && m >= 2 && !tc::mbar_wait(&aempty[b], ((m - 2) >> 1) & 1,
                                                                 abort_flag))
                            fail();
                        if (!*abort_flag) {
                            tc::tc_fence_after();
                            const uint32_t ah = tc::smem_u32(Ah), al = tc::smem_u32(Al),
                                           bh = tc::smem_u32(Bh), bl = tc::smem_u32(Bl);
                            const uint32_t dt = tmem + 32 * b;
#pragma unroll
                            for (int k = 0; k < 4; ++k) {
                                const uint64_t dah = tc::sdesc(ah + k * 32), dal = tc::sdesc(al + k * 32),
                                               dbh = tc::sdesc(bh + k * 32), dbl = tc::sdesc(bl + k * 32);
                                bos_mma_tf32(dt, dah, dbh, idesc, (kb | k) != 0);
                                bos_mma_tf32(dt, dah, dbl, idesc, 1);
                                bos_mma_tf32(dt, dal, dbh, idesc, 1);
                            }
                            tc::mma_commit(sfree);
                            if (kb == nkb - 1) tc::mma_commit(&afull[b]);
                        }
                    }
                    issue(it + 2);  // into the slot of block it, just converted
                }
                if (*abort_flag) break;
            }
            asm volatile("cp.async.wait_group 0;" ::: "memory");  // no copy outlives the block
        } else {  // epilogue warps: TMEM lanes 32 warp .. + 31 = pool entries of the tile
            for (int m = 0; m < ntile; ++m) {
                const int b = m & 1;
                int ok = 1;
                if (lane == 0) ok = tc::mbar_wait(&afull[b], (m >> 1) & 1, abort_flag) ? 1 : 0;
                ok = __shfl_sync(0xffffffffu, ok, 0);
                if (!ok) {
                    if (lane == 0) fail();
                    break;
                }
                tc::tc_fence_after();
                float w[32];
                tc::tmem_ld32(tmem + ((uint32_t)(32 * warp) << 16) + 32 * b, w);
                tc::tc_fence_before();
                __syncwarp();
                if (lane == 0) tc::mbar_arrive(&aempty[b]);
                finish(128 * m + 32 * warp + lane, w);
            }
        }
        __syncthreads();
        if (*abort_flag && tid == 128) {  // every issued MMA completes before TMEM is released
            tc::mma_commit(drain);
            tc::mbar_wait(drain, 0, nullptr);
        }
        tc::tc_fence_before();
        __syncthreads();
        if (warp == 0) {
            tc::tc_fence_after();
            asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem),
                         "r"(64));
        }
    }
    if (tid < nn) {
        d.obs[(int64_t)rp * S + s + tid] = P[tid];
        d.y[(int64_t)rp * S + s + tid] = yv[tid];
        d.beta[(int64_t)rp * S + s + tid] = b2[tid];
    }
}

__global__ void k_bos_advance(BosDev d) {
    *d.round += 1;
    d.queue[0] = 0;
    d.queue[1] = 0;
}

}  // namespace cc

// ============================================================================
// host side
using namespace cc;

struct cc_bos {
    BosDev d{};
    int field = -1, field_b = -1;
    uint64_t field_version = ~0ull, field_b_version = ~0ull;
    DevMem box, self, pool, V, mu, var, sel, obs, y, beta, hyp, prior, picks, pa, pb, vals, best,
        counters, theta, yall, inc_val, inc_idx;
    int eval_warps = 8, eval_blocks_per_sm = 4;
    bool tuned = false;
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    int rounds_done = 0;
    std::vector<int32_t> rp_a, rp_b;
};

namespace {

cc_status bfail(cc_ctx* c, cc_status s, const char* fmt, ...) {
    if (c) {
        char buf[512];
        va_list ap;
        va_start(ap, fmt);
        vsnprintf(buf, sizeof buf, fmt, ap);
        va_end(ap);
        c->err = buf;
    }
    return s;
}

#define BK(call)                                                                             \
    do {                                                                                     \
        cudaError_t _e = (call);                                                             \
        if (_e != cudaSuccess) {                                                             \
            cudaGetLastError();                                                              \
            return bfail(ctx, _e == cudaErrorMemoryAllocation ? CC_ERR_OOM : CC_ERR_CUDA,    \
                         "%s: %s", #call, cudaGetErrorString(_e));                           \
        }                                                                                    \
    } while (0)

size_t propose_smem(const BosDev& d) {
    const int M = d.M;
    return 1024 + propose_region0(d.Q) + M * 4 + (size_t)M * M * 4 + M * 6 * 4 + M * 4 + 32 * 4 +
           16 + 16;
}
size_t condition_smem(const BosDev& d) {
    const int R = d.R;
    return 1024 + kCondRegion0 + R * R * 4 + R * R * 8 + R * R * 4 + 2 * R * 4 + R * 6 * 4 +
           2 * R * 4 + 16 + (R + 1) * 4 + 6 * 8 + 16;
}
size_t eval_smem(const BosDev& d, int warps) {
    const int pl = (d.n + 2) & ~1;
    const int slots = eval_stream(d.n, d.n_pad) ? 2 : 1;
    return 2 * pl * 8 + (size_t)warps * (slots * ksg_slot_bytes(d.n_pad, ksg_kmax(d.k)) + 256 * 4);
}

// set_attr: raise the kernel's dynamic shared-memory limit first (not while
// a stream is being captured; the autotuner sets it for the largest shape).
template <int KMAX>
cudaError_t eval_launch(const BosDev& d, int warps, int blocks, bool set_attr, cudaStream_t st) {
    const size_t smem = eval_smem(d, warps);
    if (set_attr) {
        cudaError_t e = raise_smem_limit(k_bos_eval<KMAX>, smem);
        if (e != cudaSuccess) return e;
    }
    note_launch();
    k_bos_eval<KMAX><<<blocks, warps * 32, smem, st>>>(d, warps);
    return cudaGetLastError();
}

template <int KMAX>
cudaError_t eval_attr(const BosDev& d, int warps) {
    return raise_smem_limit(k_bos_eval<KMAX>, eval_smem(d, warps));
}

cudaError_t set_eval_attr(const BosDev& d, int warps) {
    const int k = d.k;
    if (k <= 1) return eval_attr<1>(d, warps);
    if (k == 2) return eval_attr<2>(d, warps);
    if (k == 3) return eval_attr<3>(d, warps);
    if (k <= 4) return eval_attr<4>(d, warps);
    if (k <= 8) return eval_attr<8>(d, warps);
    if (k <= 10) return eval_attr<10>(d, warps);
    if (k <= 16) return eval_attr<16>(d, warps);
    return eval_attr<32>(d, warps);
}

cudaError_t launch_eval(const BosDev& d, int warps, int blocks, bool set_attr, cudaStream_t st) {
    const int k = d.k;
    if (k <= 1) return eval_launch<1>(d, warps, blocks, set_attr, st);
    if (k == 2) return eval_launch<2>(d, warps, blocks, set_attr, st);
    if (k == 3) return eval_launch<3>(d, warps, blocks, set_attr, st);
    if (k <= 4) return eval_launch<4>(d, warps, blocks, set_attr, st);
    if (k <= 8) return eval_launch<8>(d, warps, blocks, set_attr, st);
    if (k <= 10) return eval_launch<10>(d, warps, blocks, set_attr, st);
    if (k <= 16) return eval_launch<16>(d, warps, blocks, set_attr, st);
    return eval_launch<32>(d, warps, blocks, set_attr, st);
}

// One round, queued on st (also the body of the captured graph).
cudaError_t enqueue_round(cc_bos* b, cudaStream_t st) {
    const BosDev& d = b->d;
    cudaError_t e;
    note_launch();
    k_bos_propose<<<d.n_rp, kBosThreads, propose_smem(d), st>>>(d);
    if ((e = cudaGetLastError())) return e;
    note_launch();
    k_bos_round_pairs<<<(d.n_rp * d.R + 255) / 256, 256, 0, st>>>(d);
    if ((e = cudaGetLastError())) return e;
    if ((e = launch_eval(d, b->eval_warps, cc::sm_count() * b->eval_blocks_per_sm, false, st)))
        return e;
    note_launch();
    k_bos_extremes<<<(4 * d.n_rp + 255) / 256, 256, 0, st>>>(d);
    if ((e = cudaGetLastError())) return e;
    note_launch();
    k_bos_condition<<<d.n_rp, kBosThreads, condition_smem(d), st>>>(d);
    if ((e = cudaGetLastError())) return e;
    note_launch();
    k_bos_advance<<<1, 1, 0, st>>>(d);
    return cudaGetLastError();
}

// Autotuner cache: "device|n|n_rp|R|k -> warps blocks_per_sm", in memory and,
// when CCORR_AUTOTUNE_CACHE names a file, as JSON lines there.
std::mutex g_tune_mu;
std::vector<std::pair<std::string, std::pair<int, int>>> g_tune;

std::string tune_key(const BosDev& d) {
    int dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceProp prop;
    cudaGetDeviceProperties(&prop, dev);
    std::ostringstream os;
    os << prop.name << "|n=" << d.n << "|rp=" << d.n_rp << "|R=" << d.R << "|k=" << d.k;
    return os.str();
}

bool tune_lookup(const std::string& key, int* w, int* b) {
    std::lock_guard<std::mutex> lock(g_tune_mu);
    for (auto& kv : g_tune)
        if (kv.first == key) {
            *w = kv.second.first;
            *b = kv.second.second;
            return true;
        }
    const char* path = getenv("CCORR_AUTOTUNE_CACHE");
    if (!path) return false;
    std::ifstream in(path);
    std::string line;
    while (std::getline(in, line)) {
        const std::string tag = "{\"key\": \"" + key + "\", ";
        if (line.rfind(tag, 0) == 0) {
            int ww = 0, bb = 0;
            if (sscanf(line.c_str() + tag.size(), "\"warps\": %d, \"blocks_per_sm\": %d", &ww,
                       &bb) == 2) {
                g_tune.push_back({key, {ww, bb}});
                *w = ww;
                *b = bb;
                return true;
            }
        }
    }
    return false;
}

void tune_store(const std::string& key, int w, int b) {
    std::lock_guard<std::mutex> lock(g_tune_mu);
    g_tune.push_back({key, {w, b}});
    const char* path = getenv("CCORR_AUTOTUNE_CACHE");
    if (!path) return;
    std::ofstream out(path, std::ios::app);
    out << "{\"key\": \"" << key << "\", \"warps\": " << w << ", \"blocks_per_sm\": " << b
        << "}\n";
}

}  // namespace

extern "C" {

cc_status cc_bos_create2(cc_ctx* ctx, int32_t field_id, int32_t field_b_id, const int32_t* rp_a,
                         const int32_t* rp_b, int n_rp, const cc_bos_params* prm, cc_bos** out) {
    if (!ctx) return CC_ERR_INVALID_ARG;
    if (!rp_a || !rp_b || !prm || !out || n_rp < 1)
        return bfail(ctx, CC_ERR_INVALID_ARG, "bad arguments");
    if (field_id < 0 || field_id >= (int)ctx->fields.size() || !ctx->fields[field_id] ||
        field_b_id < 0 || field_b_id >= (int)ctx->fields.size() || !ctx->fields[field_b_id])
        return bfail(ctx, CC_ERR_INVALID_ARG, "unknown field");
    Field& f = *ctx->fields[field_id];
    const Field& fb = *ctx->fields[field_b_id];
    if (fb.X != f.X || fb.Y != f.Y || fb.Z != f.Z || fb.n != f.n)
        return bfail(ctx, CC_ERR_INVALID_ARG,
                     "the two fields need the same grid and the same ensemble size");
    const int Q = prm->pool, R = prm->per_round, T = prm->rounds, M = prm->shortlist;
    if (Q < 256 || Q > 8192 || (Q & (Q - 1)) || R < 1 || R > 32 || T < 1 ||
        M < 16 || M > 128 || M % 16 || (int64_t)R * T + M > Q)
        return bfail(ctx, CC_ERR_INVALID_ARG,
                     "need pool a power of two in [256, 8192], 1 <= per_round <= 32, shortlist "
                     "a multiple of 16 in [16, 128], per_round * rounds + shortlist <= pool");
    if (prm->objective < CC_PEARSON || prm->objective > CC_MI_KSG)
        return bfail(ctx, CC_ERR_INVALID_ARG, "unknown objective measure");
    if (prm->local_picks < 0 || prm->local_picks >= R ||
        !(prm->local_scale > 0.f && prm->local_scale <= 1.f))
        return bfail(ctx, CC_ERR_INVALID_ARG,
                     "need 0 <= local_picks < per_round and 0 < local_scale <= 1");
    const int k = prm->k == -1 ? (3 * f.n + 99) / 100 : prm->k;
    if (k < 1 || k > f.n - 1 || k > 32 || prm->bins < 2 || prm->bins > 16)
        return bfail(ctx, CC_ERR_INVALID_ARG, "k in [1, min(n-1, 32)], bins in [2, 16]");
    std::vector<int> box(12 * n_rp), self(n_rp);
    for (int i = 0; i < n_rp; ++i) {
        const int ids[2] = {rp_a[i], rp_b[i]};
        for (int s = 0; s < 2; ++s) {
            if (ids[s] < 0 || ids[s] >= (int)ctx->regions.size() || !ctx->regions[ids[s]] ||
                ctx->regions[ids[s]]->field != (s ? field_b_id : field_id))
                return bfail(ctx, CC_ERR_INVALID_ARG, "region pair %d: bad region", i);
            const cc_box& bx = ctx->regions[ids[s]]->box;
            int* o = &box[12 * i + 6 * s];
            o[0] = bx.x0;
            o[1] = bx.y0;
            o[2] = bx.z0;
            o[3] = bx.x1 - bx.x0;
            o[4] = bx.y1 - bx.y0;
            o[5] = bx.z1 - bx.z0;
        }
        self[i] = field_id == field_b_id && rp_a[i] == rp_b[i];
        if (self[i] && box[12 * i + 3] * box[12 * i + 4] * box[12 * i + 5] < 2)
            return bfail(ctx, CC_ERR_INVALID_ARG, "self pair needs two points");
    }
    cc_bos* b = new (std::nothrow) cc_bos();
    if (!b) return CC_ERR_OOM;
    std::unique_ptr<cc_bos> guard(b);
    b->field = field_id;
    b->field_b = field_b_id;
    b->rp_a.assign(rp_a, rp_a + n_rp);
    b->rp_b.assign(rp_b, rp_b + n_rp);
    BosDev& d = b->d;
    d.n_rp = n_rp;
    d.Q = Q;
    d.R = R;
    d.T = T;
    d.M = M;
    d.L = prm->local_picks;
    d.lscale = prm->local_scale;
    d.S = R + (T - 1) * (R - d.L);
    d.Sp = (d.S + 7) / 8 * 8;
    d.kappa = prm->kappa;
    d.seed = prm->seed;
    d.objective = prm->objective;
    d.k = k;
    d.bins = prm->bins;
    d.n = f.n;
    d.n_pad = f.n_pad;
    d.X = f.X;
    d.Y = f.Y;
    const int64_t S = d.S, RT = (int64_t)R * T;
    BK(b->box.alloc(box.size() * 4));
    BK(b->self.alloc(self.size() * 4));
    BK(b->pool.alloc((size_t)n_rp * Q * 6 * 4));
    BK(b->V.alloc((size_t)n_rp * Q * d.Sp * 4));
    BK(b->mu.alloc((size_t)n_rp * Q * 4));
    BK(b->var.alloc((size_t)n_rp * Q * 4));
    BK(b->sel.alloc((size_t)n_rp * (Q / 32) * 4));
    BK(b->obs.alloc((size_t)n_rp * S * 4));
    BK(b->y.alloc((size_t)n_rp * S * 4));
    BK(b->beta.alloc((size_t)n_rp * S * 4));
    BK(b->hyp.alloc((size_t)n_rp * 4 * 4));
    BK(b->picks.alloc((size_t)n_rp * R * 4));
    BK(b->pa.alloc((size_t)n_rp * R * 4));
    BK(b->pb.alloc((size_t)n_rp * R * 4));
    BK(b->vals.alloc((size_t)4 * n_rp * R * 4));
    BK(b->best.alloc((size_t)4 * n_rp * sizeof(Partial)));
    BK(b->counters.alloc(16));
    BK(b->theta.alloc((size_t)n_rp * RT * 6 * 4));
    BK(b->yall.alloc((size_t)n_rp * RT * 4));
    BK(b->inc_val.alloc((size_t)n_rp * 2 * 4));
    BK(b->inc_idx.alloc((size_t)n_rp * 2 * 4));
    cudaStream_t st = ctx->stream;
    BK(cudaMemcpyAsync(b->box.p, box.data(), box.size() * 4, cudaMemcpyHostToDevice, st));
    BK(cudaMemcpyAsync(b->self.p, self.data(), self.size() * 4, cudaMemcpyHostToDevice, st));
    BK(cudaMemsetAsync(b->sel.p, 0, b->sel.bytes, st));
    BK(cudaMemsetAsync(b->counters.p, 0, 16, st));
    BK(cudaMemsetAsync(b->beta.p, 0, b->beta.bytes, st));
    BK(cudaMemsetAsync(b->V.p, 0, b->V.bytes, st));  // rows not yet written read as zero
    d.box = b->box.as<int>();
    d.self = b->self.as<int>();
    d.pool = b->pool.as<float>();
    d.V = b->V.as<float>();
    d.mu = b->mu.as<float>();
    d.var = b->var.as<float>();
    d.sel = b->sel.as<unsigned>();
    d.obs = b->obs.as<int>();
    d.y = b->y.as<float>();
    d.beta = b->beta.as<float>();
    d.hyp = b->hyp.as<float>();
    d.theta = b->theta.as<float>();
    d.yall = b->yall.as<float>();
    d.inc_val = b->inc_val.as<float>();
    d.inc_idx = b->inc_idx.as<int>();
    d.prior = nullptr;
    d.picks = b->picks.as<int>();
    d.pa = b->pa.as<uint32_t>();
    d.pb = b->pb.as<uint32_t>();
    d.vals = b->vals.as<float>();
    d.best = b->best.as<Partial>();
    d.round = b->counters.as<int>();
    d.queue = b->counters.as<int>() + 1;
    d.status = ctx->status.as<int>();
    note_launch();
    k_bos_pool<<<(unsigned)(((int64_t)n_rp * Q + 255) / 256), 256, 0, st>>>(d);
    BK(cudaGetLastError());
    BK(raise_smem_limit(k_bos_propose, propose_smem(d)));
    BK(raise_smem_limit(k_bos_condition, condition_smem(d)));
    BK(cudaStreamSynchronize(st));
    *out = guard.release();
    return CC_OK;
}

cc_status cc_bos_create(cc_ctx* ctx, int32_t field_id, const int32_t* rp_a, const int32_t* rp_b,
                        int n_rp, const cc_bos_params* prm, cc_bos** out) {
    return cc_bos_create2(ctx, field_id, field_id, rp_a, rp_b, n_rp, prm, out);
}

cc_status cc_bos_set_prior(cc_ctx* ctx, cc_bos* b, const float* prior, int prior_is_device) {
    if (!ctx || !b) return CC_ERR_INVALID_ARG;
    if (b->rounds_done > 0)
        return bfail(ctx, CC_ERR_INVALID_ARG, "the prior must be set before the first round");
    if (!prior) {
        b->d.prior = nullptr;
        return CC_OK;
    }
    const size_t bytes = (size_t)b->d.n_rp * b->d.Q * 4;
    BK(b->prior.alloc(bytes));
    BK(cudaMemcpyAsync(b->prior.p, prior, bytes,
                       prior_is_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice,
                       ctx->stream));
    b->d.prior = b->prior.as<float>();
    if (b->exec) {  // the captured graph holds the old parameters
        cudaGraphExecDestroy(b->exec);
        cudaGraphDestroy(b->graph);
        b->exec = nullptr;
        b->graph = nullptr;
    }
    return CC_OK;
}

cc_status cc_bos_run(cc_ctx* ctx, cc_bos* b, int rounds, int use_graph) {
    if (!ctx || !b || rounds < 0) return CC_ERR_INVALID_ARG;
    if (b->rounds_done + rounds > b->d.T)
        return bfail(ctx, CC_ERR_INVALID_ARG, "only %d rounds were provisioned", b->d.T);
    if (b->field >= (int)ctx->fields.size() || !ctx->fields[b->field] ||
        b->field_b >= (int)ctx->fields.size() || !ctx->fields[b->field_b])
        return bfail(ctx, CC_ERR_INVALID_ARG, "a field of this search was freed");
    Field& f = *ctx->fields[b->field];
    Field& fb = *ctx->fields[b->field_b];
    // field planes (bins for the binned measure, tables) are bound at the first round
    if (b->field_version != f.version || b->field_b_version != fb.version) {
        if (b->rounds_done > 0)
            return bfail(ctx, CC_ERR_INVALID_ARG, "the field changed during sampling");
        cc_params p{CC_MI_BINNED, b->d.k, b->d.bins, 0, 0};
        // evaluate one in-range pair so the bins and tables of both fields exist
        uint32_t one = 0;
        float tmp = 0.f;
        cc_status s = cc_eval_pairs(ctx, b->field, b->field_b, &p, &one, &one, 1, 0, &tmp, 0);
        if (s) return s;
        p.measure = CC_MI_KSG;
        if ((s = cc_eval_pairs(ctx, b->field, b->field_b, &p, &one, &one, 1, 0, &tmp, 0)))
            return s;
        b->d.zhat = f.zhat.as<float>();
        b->d.rhat = f.rhat.as<float>();
        b->d.fvals = f.vals.as<float>();
        b->d.sorted = f.sorted.as<float>();
        b->d.perm = f.perm.as<uint16_t>();
        b->d.bins_p = f.bins[b->d.bins]->as<uint8_t>();
        b->d.hmarg = (const long long*)f.hmarg[b->d.bins]->as<int64_t>();
        b->d.zhat_b = fb.zhat.as<float>();
        b->d.rhat_b = fb.rhat.as<float>();
        b->d.fvals_b = fb.vals.as<float>();
        b->d.sorted_b = fb.sorted.as<float>();
        b->d.perm_b = fb.perm.as<uint16_t>();
        b->d.bins_b = fb.bins[b->d.bins]->as<uint8_t>();
        b->d.hmarg_b = (const long long*)fb.hmarg[b->d.bins]->as<int64_t>();
        b->d.psi_fix = (const long long*)ctx->psi_fix[f.n]->as<int64_t>();
        b->d.clogc_fix = (const long long*)ctx->clogc_fix[f.n]->as<int64_t>();
        b->d.psi_nk = digamma_int_host(f.n) + digamma_int_host(b->d.k);
        b->d.fix_over_n = 1.0 / (kFixScale * f.n);
        b->d.logn = std::log((double)f.n);
        b->field_version = f.version;
        b->field_b_version = fb.version;
    }
    cudaStream_t st = ctx->stream;
    if (!b->tuned) {
        const std::string key = tune_key(b->d);
        int w = 8, bps = 4;
        if (!tune_lookup(key, &w, &bps)) {
            // time the evaluation on the first round's proposals for each shape
            note_launch(2);
            k_bos_propose<<<b->d.n_rp, kBosThreads, propose_smem(b->d), st>>>(b->d);
            k_bos_round_pairs<<<(b->d.n_rp * b->d.R + 255) / 256, 256, 0, st>>>(b->d);
            BK(cudaGetLastError());
            float best_ms = 1e30f;
            cudaEvent_t e0, e1;
            BK(cudaEventCreate(&e0));
            BK(cudaEventCreate(&e1));
            const int shapes[6][2] = {{4, 4}, {4, 8}, {8, 2}, {8, 4}, {16, 1}, {16, 2}};
            for (auto& sh : shapes) {
                float ms = 0.f;
                for (int rep = 0; rep < 2; ++rep) {
                    BK(cudaMemsetAsync(b->d.queue, 0, 8, st));
                    BK(cudaEventRecord(e0, st));
                    BK(launch_eval(b->d, sh[0], cc::sm_count() * sh[1], true, st));
                    BK(cudaEventRecord(e1, st));
                    BK(cudaEventSynchronize(e1));
                    BK(cudaEventElapsedTime(&ms, e0, e1));
                }
                if (ms < best_ms) {
                    best_ms = ms;
                    w = sh[0];
                    bps = sh[1];
                }
            }
            cudaEventDestroy(e0);
            cudaEventDestroy(e1);
            BK(cudaMemsetAsync(b->d.queue, 0, 8, st));
            tune_store(key, w, bps);
        }
        b->eval_warps = w;
        b->eval_blocks_per_sm = bps;
        BK(set_eval_attr(b->d, w));
        b->tuned = true;
    }
    for (int r = 0; r < rounds; ++r) {
        if (use_graph) {
            if (!b->exec) {
                BK(cudaStreamBeginCapture(st, cudaStreamCaptureModeThreadLocal));
                cudaError_t e = enqueue_round(b, st);
                cudaGraph_t g = nullptr;
                cudaError_t e2 = cudaStreamEndCapture(st, &g);
                if (e != cudaSuccess || e2 != cudaSuccess) {
                    if (g) cudaGraphDestroy(g);
                    cudaGetLastError();
                    return bfail(ctx, CC_ERR_CUDA, "graph capture failed: %s",
                                 cudaGetErrorString(e ? e : e2));
                }
                b->graph = g;
                BK(cudaGraphInstantiate(&b->exec, g, 0));
            }
            note_launch(6);
            BK(cudaGraphLaunch(b->exec, st));
        } else {
            BK(enqueue_round(b, st));
        }
        b->rounds_done++;
    }
    return CC_OK;
}

cc_status cc_bos_results(cc_ctx* ctx, cc_bos* b, cc_rp_result* out) {
    if (!ctx || !b || !out) return CC_ERR_INVALID_ARG;
    std::vector<Partial> h(4 * (size_t)b->d.n_rp);
    BK(cudaMemcpyAsync(h.data(), b->best.p, h.size() * sizeof(Partial), cudaMemcpyDeviceToHost,
                       ctx->stream));
    BK(cudaStreamSynchronize(ctx->stream));
    for (size_t i = 0; i < h.size(); ++i)
        out[i] = cc_rp_result{h[i].max, h[i].min, h[i].argmax, h[i].argmin, h[i].count};
    return CC_OK;
}

cc_status cc_bos_inspect(cc_ctx* ctx, cc_bos* b, int rp, float* pool, float* mu, float* var,
                         int32_t* obs, float* y, uint32_t* pa, uint32_t* pb, float* vals,
                         int32_t* n_obs) {
    if (!ctx || !b || rp < 0 || rp >= b->d.n_rp) return CC_ERR_INVALID_ARG;
    const BosDev& d = b->d;
    const int64_t S = d.S, s = obs_before(b->rounds_done, d.R, d.L);
    cudaStream_t st = ctx->stream;
    if (pool) BK(cudaMemcpyAsync(pool, d.pool + (int64_t)rp * d.Q * 6, d.Q * 24, cudaMemcpyDeviceToHost, st));
    if (mu) BK(cudaMemcpyAsync(mu, d.mu + (int64_t)rp * d.Q, d.Q * 4, cudaMemcpyDeviceToHost, st));
    if (var) BK(cudaMemcpyAsync(var, d.var + (int64_t)rp * d.Q, d.Q * 4, cudaMemcpyDeviceToHost, st));
    if (obs && s) BK(cudaMemcpyAsync(obs, d.obs + rp * S, s * 4, cudaMemcpyDeviceToHost, st));
    if (y && s) BK(cudaMemcpyAsync(y, d.y + rp * S, s * 4, cudaMemcpyDeviceToHost, st));
    if (pa) BK(cudaMemcpyAsync(pa, d.pa + rp * d.R, d.R * 4, cudaMemcpyDeviceToHost, st));
    if (pb) BK(cudaMemcpyAsync(pb, d.pb + rp * d.R, d.R * 4, cudaMemcpyDeviceToHost, st));
    if (vals)
        for (int m = 0; m < 4; ++m)
            BK(cudaMemcpyAsync(vals + m * d.R, d.vals + (int64_t)m * d.n_rp * d.R + rp * d.R,
                               d.R * 4, cudaMemcpyDeviceToHost, st));
    if (n_obs) *n_obs = (int32_t)s;
    BK(cudaStreamSynchronize(st));
    return CC_OK;
}

cc_status cc_bos_samples(cc_ctx* ctx, cc_bos* b, int rp, float* theta, float* y,
                         int32_t* n_samples) {
    if (!ctx || !b || rp < 0 || rp >= b->d.n_rp) return CC_ERR_INVALID_ARG;
    const BosDev& d = b->d;
    const int64_t RT = (int64_t)d.R * d.T, n = (int64_t)b->rounds_done * d.R;
    cudaStream_t st = ctx->stream;
    if (theta && n)
        BK(cudaMemcpyAsync(theta, d.theta + rp * RT * 6, n * 24, cudaMemcpyDeviceToHost, st));
    if (y && n) BK(cudaMemcpyAsync(y, d.yall + rp * RT, n * 4, cudaMemcpyDeviceToHost, st));
    if (n_samples) *n_samples = (int32_t)n;
    BK(cudaStreamSynchronize(st));
    return CC_OK;
}

cc_status cc_bos_destroy(cc_ctx* ctx, cc_bos* b) {
    if (!b) return CC_ERR_INVALID_ARG;
    if (ctx) cudaStreamSynchronize(ctx->stream);
    if (b->exec) cudaGraphExecDestroy(b->exec);
    if (b->graph) cudaGraphDestroy(b->graph);
    delete b;
    return CC_OK;
}

}  // extern "C"
