// Learned pairwise surrogate (project addition; the paper's Section 7 names
// a network predicting MI as future work): BF16 training and inference.
//
//   encoder  z (n) -> h1 = GELU(W1 z + b1) (128) -> e = W2 h1 + b2 (64)
//   head     x = [e_i, e_j, |e_i - e_j|, off] (195) -> h3 = GELU(W3 x + b3)
//            (128) -> y = w4 . h3 + b4
// z = zhat * sqrt(n - 1) (the member vector's z-score), off = position
// difference / field size, GELU in the erf form. MSE on standardized targets,
// Adam (beta 0.9 / 0.999, eps 1e-8) on fp32 master weights; GEMM inputs are
// BF16 (weights and activations) or fp32 (back-propagated gradients), all
// accumulation fp32. Parameters are one flat fp32 vector: W1 (128 x n), b1,
// W2 (64 x 128), b2, W3 (128 x 195), b3, w4 (128), b4.
//
// The all-pairs screen splits the head's first layer: W3 x = Wa e_i + Wb e_j
// + Wc |e_i - e_j| + Wd off, with Wa e_i and Wb e_j computed once per point,
// so a pair costs the 128 x 64 contraction of |e_i - e_j| plus 128 GELUs.
#include <cuda_bf16.h>
#include <math.h>
#include <stdarg.h>
#include <stdio.h>

#include <algorithm>
#include <thread>
#include <type_traits>
#include <vector>

#include "device.cuh"
#include "internal.cuh"

namespace cc {

constexpr int kH1 = 128, kE = 64, kH3 = 128, kHeadIn = 3 * kE + 3;
// row strides of the BF16 GEMM operands padded to 16 bytes (the tensor-core
// GEMM then reads whole 16-byte chunks): encoder inputs and W1 rows of n
// values, head inputs and W3 rows of 195
constexpr int kHeadInP = 200;
__host__ __device__ inline int ldz(int n) { return (n + 7) & ~7; }

// padded BF16 copies of W1 [128][ldz(n)] and W3 [128][kHeadInP], written
// wherever the BF16 weight vector is written
struct PadW {
    __nv_bfloat16* p;
    int64_t oW1, oW3;
    int n;
};
__device__ __forceinline__ void pad_store(const PadW& pw, int64_t i, __nv_bfloat16 v) {
    if (i >= pw.oW1 && i < pw.oW1 + (int64_t)kH1 * pw.n) {
        const int64_t j = i - pw.oW1;
        pw.p[(j / pw.n) * ldz(pw.n) + j % pw.n] = v;
    } else if (i >= pw.oW3 && i < pw.oW3 + (int64_t)kH3 * kHeadIn) {
        const int64_t j = i - pw.oW3;
        pw.p[(int64_t)kH1 * ldz(pw.n) + (j / kHeadIn) * kHeadInP + j % kHeadIn] = v;
    }
}

struct SurOff {
    int64_t W1, b1, W2, b2, W3, b3, w4, b4, total;
    explicit SurOff(int n) {
        W1 = 0;
        b1 = W1 + (int64_t)kH1 * n;
        W2 = b1 + kH1;
        b2 = W2 + (int64_t)kE * kH1;
        W3 = b2 + kE;
        b3 = W3 + (int64_t)kH3 * kHeadIn;
        w4 = b3 + kH3;
        b4 = w4 + kH3;
        total = b4 + 1;
    }
};

__device__ __forceinline__ float ld(const float* p) { return *p; }
__device__ __forceinline__ float ld(const __nv_bfloat16* p) { return __bfloat162float(*p); }

__device__ __forceinline__ float gelu(float x) {
    return 0.5f * x * (1.f + erff(x * 0.70710678118654752f));
}
__device__ __forceinline__ float gelu_grad(float x) {
    return 0.5f * (1.f + erff(x * 0.70710678118654752f)) +
           x * expf(-0.5f * x * x) * 0.39894228040143268f;
}

// Generic strided GEMM C (+)= A B with A[m][k] = A[m * sam + k * sak] and
// B[k][n] = B[k * sbk + n * sbn] (fp32 or bf16 inputs, fp32 accumulation).
// 64 x 64 output tile per CTA, 256 threads with 4 x 4 outputs, K staged 16 at
// a time through shared memory; each operand tile is read along its
// unit-stride dimension. Split-K over gridDim.z: slice z covers k in
// [z kc, (z + 1) kc) and writes a dense partial [M][N] that k_mm_reduce sums
// in slice order (deterministic), so the weight gradients (M x N small, K =
// the batch) still fill the GPU.
template <class TA, class TB>
__global__ void __launch_bounds__(256)
    k_mm(const TA* __restrict__ A, int64_t sam, int64_t sak, const TB* __restrict__ B,
         int64_t sbk, int64_t sbn, float* __restrict__ C, int64_t ldc, int M, int N, int K,
         int kc, int accumulate, float* __restrict__ part) {
    __shared__ float As[16][64 + 1];
    __shared__ float Bs[16][64 + 1];
    const int tid = threadIdx.x, tx = tid & 15, ty = tid >> 4;
    const int m0 = blockIdx.y * 64, n0 = blockIdx.x * 64;
    const int kb = blockIdx.z * kc, ke = min(K, kb + kc);
    const bool a_k = sak == 1, b_k = sbk == 1;
    float acc[4][4] = {};
    for (int k0 = kb; k0 < ke; k0 += 16) {
        for (int e = tid; e < 16 * 64; e += 256) {
            const int kk = a_k ? (e & 15) : (e >> 6), mm = a_k ? (e >> 4) : (e & 63);
            const int m = m0 + mm, k = k0 + kk;
            As[kk][mm] = (m < M && k < ke) ? ld(A + m * sam + k * sak) : 0.f;
        }
        for (int e = tid; e < 16 * 64; e += 256) {
            const int kk = b_k ? (e & 15) : (e >> 6), nn = b_k ? (e >> 4) : (e & 63);
            const int n = n0 + nn, k = k0 + kk;
            Bs[kk][nn] = (n < N && k < ke) ? ld(B + k * sbk + n * sbn) : 0.f;
        }
        __syncthreads();
#pragma unroll
        for (int kk = 0; kk < 16; ++kk) {
            float a[4], b[4];
#pragma unroll
            for (int i = 0; i < 4; ++i) a[i] = As[kk][ty + 16 * i];
#pragma unroll
            for (int j = 0; j < 4; ++j) b[j] = Bs[kk][tx + 16 * j];
#pragma unroll
            for (int i = 0; i < 4; ++i)
#pragma unroll
                for (int j = 0; j < 4; ++j) acc[i][j] = fmaf(a[i], b[j], acc[i][j]);
        }
        __syncthreads();
    }
#pragma unroll
    for (int i = 0; i < 4; ++i) {
        const int m = m0 + ty + 16 * i;
        if (m >= M) continue;
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            const int n = n0 + tx + 16 * j;
            if (n >= N) continue;
            if (part) {
                part[((int64_t)blockIdx.z * M + m) * N + n] = acc[i][j];
            } else {
                float* c = C + (int64_t)m * ldc + n;
                *c = accumulate ? *c + acc[i][j] : acc[i][j];
            }
        }
    }
}

// C = the sum of S dense partials [S][M][N]: slice z adds into accumulator
// z mod 8 and the eight are added in order (a fixed order, so the result does
// not depend on timing). A block of 256 threads takes 32 outputs: warp j sums
// the slices z = j mod 8 of its lane's output, so every output's eight
// accumulators are summed in parallel. With bias, column N - 1 goes to
// bias[m] and C receives columns 0 .. N - 2.
constexpr int kReduceOuts = 32;  // outputs per block of k_mm_reduce (256 threads)
__global__ void __launch_bounds__(256)
    k_mm_reduce(const float* __restrict__ part, int S, int M, int N, float* __restrict__ C,
                int64_t ldc, int accumulate, float* __restrict__ bias) {
    __shared__ float red[8][kReduceOuts + 1];
    const int64_t MN = (int64_t)M * N;
    const int lane = threadIdx.x & 31, j = threadIdx.x >> 5;
    const int64_t e = (int64_t)blockIdx.x * kReduceOuts + lane;
    float a = 0.f;
    if (e < MN)
        for (int z = j; z < S; z += 8) a += part[(int64_t)z * MN + e];
    red[j][lane] = a;
    __syncthreads();
    if (j == 0 && e < MN) {
        const float s = ((red[0][lane] + red[1][lane]) + (red[2][lane] + red[3][lane])) +
                        ((red[4][lane] + red[5][lane]) + (red[6][lane] + red[7][lane]));
        const int64_t m = e / N;
        const int n = (int)(e % N);
        if (bias && n == N - 1) {
            bias[m] = accumulate ? bias[m] + s : s;
        } else {
            float* c = C + m * ldc + n;
            *c = accumulate ? *c + s : s;
        }
    }
}
inline unsigned reduce_blocks(int64_t MN) { return (unsigned)((MN + kReduceOuts - 1) / kReduceOuts); }

// Up to four k_mm_reduce problems in one launch (a training step's weight
// gradients, each from its own partials): block b belongs to the segment
// whose range of reduce_blocks holds b, and reduces its 32 outputs in the
// same order as k_mm_reduce (accumulate = 0).
struct ReduceSeg {
    const float* part = nullptr;
    int S = 0, M = 0, N = 0;
    float* C = nullptr;
    int64_t ldc = 0;
    float* bias = nullptr;
    unsigned blocks = 0;  // reduce_blocks(M N); 0: nothing to reduce
};
struct ReduceSegs {
    ReduceSeg s[4];
};
__global__ void __launch_bounds__(256) k_mm_reduce_multi(ReduceSegs segs) {
    __shared__ float red[8][kReduceOuts + 1];
    unsigned blk = blockIdx.x;
    int q = 0;
    while (q < 3 && blk >= segs.s[q].blocks) blk -= segs.s[q++].blocks;  // block-uniform
    const ReduceSeg g = segs.s[q];
    const int64_t MN = (int64_t)g.M * g.N;
    const int lane = threadIdx.x & 31, j = threadIdx.x >> 5;
    const int64_t e = (int64_t)blk * kReduceOuts + lane;
    float a = 0.f;
    if (e < MN)
        for (int z = j; z < g.S; z += 8) a += g.part[(int64_t)z * MN + e];
    red[j][lane] = a;
    __syncthreads();
    if (j == 0 && e < MN) {
        const float sum = ((red[0][lane] + red[1][lane]) + (red[2][lane] + red[3][lane])) +
                          ((red[4][lane] + red[5][lane]) + (red[6][lane] + red[7][lane]));
        const int64_t m = e / g.N;
        const int n = (int)(e % g.N);
        if (g.bias && n == g.N - 1) g.bias[m] = sum;
        else g.C[m * g.ldc + n] = sum;
    }
}

template <class TA, class TB>
static cudaError_t mm(const TA* A, int64_t sam, int64_t sak, const TB* B, int64_t sbk, int64_t sbn,
                      float* C, int64_t ldc, int M, int N, int K, int acc, cudaStream_t st,
                      DevMem* ws = nullptr) {
    const int gx = (N + 63) / 64, gy = (M + 63) / 64;
    // split K when the output tiles alone would leave most SMs idle
    int S = 1, kc = ((K + 15) / 16) * 16;
    const int sms = sm_count();
    if (ws && gx * gy < sms && K >= 512) {
        S = std::min((2 * sms + gx * gy - 1) / (gx * gy), K / 128);
        kc = ((K + S - 1) / S + 15) / 16 * 16;
        S = (K + kc - 1) / kc;
        cudaError_t e = ws->ensure(sizeof(float) * (size_t)S * M * N);
        if (e != cudaSuccess) return e;
    }
    note_launch();
    k_mm<TA, TB><<<dim3(gx, gy, S), 256, 0, st>>>(A, sam, sak, B, sbk, sbn, C, ldc, M, N, K, kc,
                                                  acc, S > 1 ? ws->as<float>() : nullptr);
    if (S > 1) {
        note_launch();
        const int64_t MN = (int64_t)M * N;
        k_mm_reduce<<<reduce_blocks(MN), 256, 0, st>>>(ws->as<float>(), S, M, N, C, ldc, acc,
                                                        nullptr);
    }
    return cudaGetLastError();
}

// The same product on the tensor cores (tc_mm.cu) when N <= 256 and the
// operands are 16-byte aligned along a unit-stride dimension, with the
// arguments in mm's order; weight gradients (few output tiles, K = the
// batch) split K into slices of at least 128 and sum the slices' partials in
// slice order. Otherwise (e.g. encoders of more than 256 members) k_mm.
__global__ void k_sur_colsum(const float* __restrict__ A, int64_t rows, int cols,
                             float* __restrict__ out);

template <class TA, class TB>
static cudaError_t tmm(int* status, const TA* A, int64_t sam, int64_t sak, const TB* B,
                       int64_t sbk, int64_t sbn, float* C, int64_t ldc, int M, int N, int K,
                       cudaStream_t st, DevMem* ws = nullptr, float* bias = nullptr,
                       ReduceSeg* defer = nullptr) {
    // bias (weight gradients): bias[m] = sum_k A(m, k), A an FP32 [K][M] matrix,
    // computed as one more output column against an all-ones row of B.
    // defer: the split-K partials' reduction is described in *defer for one
    // later k_mm_reduce_multi launch instead of launched here (blocks 0: none)
    if (defer) *defer = ReduceSeg{};
    const int NB = N + (bias ? 1 : 0);
    auto fallback = [&]() -> cudaError_t {
        cudaError_t e = mm(A, sam, sak, B, sbk, sbn, C, ldc, M, N, K, 0, st, ws);
        if (e != cudaSuccess || !bias) return e;
        note_launch();
        k_sur_colsum<<<M, 256, 0, st>>>(reinterpret_cast<const float*>(A), K, M, bias);
        return cudaGetLastError();
    };
    if (NB > 256) return fallback();
    constexpr int abf = std::is_same<TA, __nv_bfloat16>::value;
    constexpr int bbf = std::is_same<TB, __nv_bfloat16>::value;
    if (bias && (abf || sam != 1 || sak != M)) return cudaErrorInvalidValue;
    const int64_t mt = (M + 127) / 128;
    const int sms = sm_count();
    int64_t kc = ((int64_t)K + 63) / 64 * 64, S = 1;
    if (ws && 2 * mt < sms && K >= 1024) {
        S = std::max<int64_t>(1, std::min<int64_t>(sms / mt, K / 128));
        kc = ((K + S - 1) / S + 63) / 64 * 64;
        S = (K + kc - 1) / kc;
    }
    if (S == 1 && !bias) {
        const cudaError_t e = launch_tc_mm(A, abf, sam, sak, B, bbf, sbn, sbk, -1, C, ldc, M, N, K,
                                           kc, nullptr, status, st);
        return e == cudaErrorNotSupported ? fallback() : e;
    }
    if (!ws) return cudaErrorInvalidValue;
    cudaError_t e = ws->ensure(sizeof(float) * (size_t)S * M * NB);
    if (e != cudaSuccess) return e;
    e = launch_tc_mm(A, abf, sam, sak, B, bbf, sbn, sbk, bias ? N : -1, nullptr, NB, M, NB, K, kc,
                     ws->as<float>(), status, st);
    if (e == cudaErrorNotSupported) return fallback();
    if (e != cudaSuccess) return e;
    const int64_t MN = (int64_t)M * NB;
    if (defer) {
        *defer = ReduceSeg{ws->as<float>(), (int)S, M, NB, C, ldc, bias, reduce_blocks(MN)};
        return cudaSuccess;
    }
    note_launch();
    k_mm_reduce<<<reduce_blocks(MN), 256, 0, st>>>(ws->as<float>(), (int)S, M, NB, C, ldc, 0,
                                                    bias);
    return cudaGetLastError();
}

// Gradients of the output layer: partial sums over a chunk of 64 rows per
// block, part[i][h] = sum_b H3[b][h] dy[b] (h < 128) and part[i][128] =
// sum_b dy[b] (b4); k_mm_reduce adds the chunks into w4 and b4 (adjacent).
__global__ void k_sur_w4_grad(const __nv_bfloat16* __restrict__ H3, const float* __restrict__ dy,
                              int64_t B, float* __restrict__ part) {
    const int64_t b0 = (int64_t)blockIdx.x * 64, b1 = min(B, b0 + 64);
    const int h = threadIdx.x;
    float* out = part + (int64_t)blockIdx.x * (kH3 + 1);
    if (h < kH3) {
        float s = 0.f;
        for (int64_t b = b0; b < b1; ++b) s = fmaf(__bfloat162float(H3[b * kH3 + h]), dy[b], s);
        out[h] = s;
    } else if (h < kH3 + 32) {
        float s = 0.f;
        for (int64_t b = b0 + (h - kH3); b < b1; b += 32) s += dy[b];
        s = warp_sum_f32(s);
        if (h == kH3) out[kH3] = s;
    }
}

// ---------------------------------------------------------------------------
// encoder inputs: row r of X0 = z-scores of point pts[r] (bf16)
__global__ void k_sur_gather_z(const float* __restrict__ zhat, int n, int n_pad, float scale,
                               const uint32_t* __restrict__ pts, int64_t rows, int ldx,
                               __nv_bfloat16* __restrict__ X0) {
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < rows * n;
         e += (int64_t)gridDim.x * blockDim.x) {
        const int64_t r = e / n;
        const int k = (int)(e % n);
        X0[r * ldx + k] = __float2bfloat16_rn(zhat[(int64_t)pts[r] * n_pad + k] * scale);
    }
}

// act = GELU(pre + bias) (bf16), pre keeps the pre-activation (fp32)
__global__ void k_sur_bias_gelu(float* __restrict__ pre, const float* __restrict__ bias, int64_t rows,
                                int cols, __nv_bfloat16* __restrict__ act) {
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < rows * cols;
         e += (int64_t)gridDim.x * blockDim.x) {
        const float a = pre[e] + bias[e % cols];
        pre[e] = a;
        act[e] = __float2bfloat16_rn(gelu(a));
    }
}

// head input x = [e_i, e_j, |e_i - e_j|, off]; encoder rows 0..B-1 hold i,
// rows B..2B-1 hold j
__global__ void k_sur_head_input(const float* __restrict__ Ef, const float* __restrict__ b2,
                                 const uint32_t* __restrict__ pi, const uint32_t* __restrict__ pj,
                                 int X, int Y, int Z, int64_t B, __nv_bfloat16* __restrict__ X3,
                                 float* __restrict__ Eout) {
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < B * kHeadIn;
         e += (int64_t)gridDim.x * blockDim.x) {
        const int64_t b = e / kHeadIn;
        const int c = (int)(e % kHeadIn);
        float v;
        if (c < 3 * kE) {
            const int q = c % kE;
            const float ei = Ef[b * kE + q] + b2[q];
            const float ej = Ef[(B + b) * kE + q] + b2[q];
            if (c < kE) {
                v = ei;
                Eout[b * kE + q] = ei;
                Eout[(B + b) * kE + q] = ej;
            } else {
                v = c < 2 * kE ? ej : fabsf(ei - ej);
            }
        } else {
            const int a = c - 3 * kE;
            const int64_t p = pi[b], q = pj[b];
            const int64_t dp = a == 0 ? (q % X) - (p % X)
                               : a == 1 ? ((q / X) % Y) - ((p / X) % Y)
                                        : (q / ((int64_t)X * Y)) - (p / ((int64_t)X * Y));
            v = (float)dp / (float)(a == 0 ? X : a == 1 ? Y : Z);
        }
        X3[b * kHeadInP + c] = __float2bfloat16_rn(v);
    }
}

// y = w4 . h3 + b4; loss terms and dy = 2 (y - t) / B (one warp per row, 256 threads)
// with t, also the head's GELU backward dA3[b][h] = (dy[b] w4[h]) gelu'(A3[b][h])
__global__ void k_sur_out(const __nv_bfloat16* __restrict__ H3, const float* __restrict__ w4,
                          const float* __restrict__ b4, const float* __restrict__ t, int64_t B,
                          float tmean, float tinv, float* __restrict__ y, float* __restrict__ dy,
                          double* __restrict__ loss, const float* __restrict__ A3,
                          float* __restrict__ dA3) {
    __shared__ double block_loss[8];  // 256 threads
    const int lane = threadIdx.x & 31;
    double wloss = 0.0;  // this warp's rows' squared residuals (lane 0)
    for (int64_t b = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5; b < B;
         b += ((int64_t)gridDim.x * blockDim.x) >> 5) {
        float s = 0.f;
        for (int h = lane; h < kH3; h += 32) s = fmaf(__bfloat162float(H3[b * kH3 + h]), w4[h], s);
        s = warp_sum_f32(s) + b4[0];
        float d = 0.f;
        if (lane == 0) {
            y[b] = s;
            if (t) {
                const float r = s - (t[b] - tmean) * tinv;
                d = 2.f * r / (float)B;
                dy[b] = d;
                wloss += (double)r * r;
            }
        }
        if (t) {
            d = __shfl_sync(0xffffffffu, d, 0);
            for (int h = lane; h < kH3; h += 32)
                dA3[b * kH3 + h] = (d * w4[h]) * gelu_grad(A3[b * kH3 + h]);
        }
    }
    if (t) {  // one atomic per block on the loss (one address for every row)
        if (lane == 0) block_loss[threadIdx.x >> 5] = wloss;
        __syncthreads();
        if (threadIdx.x == 0) {
            double l = 0.0;
            for (int w = 0; w < (int)(blockDim.x >> 5); ++w) l += block_loss[w];
            atomicAdd(loss, l);
        }
    }
}

// dA = (dy outer w4) * gelu'(pre)   (head) or dA = dH * gelu'(pre) (encoder)
__global__ void k_sur_gelu_bwd(const float* __restrict__ pre, const float* __restrict__ dy,
                               const float* __restrict__ w4, const float* __restrict__ dH,
                               int64_t rows, int cols, float* __restrict__ dA) {
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < rows * cols;
         e += (int64_t)gridDim.x * blockDim.x) {
        const float g = dH ? dH[e] : dy[e / cols] * w4[e % cols];
        dA[e] = g * gelu_grad(pre[e]);
    }
}

// column sums of a [rows][cols] fp32 matrix into out (one block per column)
__global__ void k_sur_colsum(const float* __restrict__ A, int64_t rows, int cols,
                             float* __restrict__ out) {
    __shared__ float red[256];
    const int c = blockIdx.x;
    float s = 0.f;
    for (int64_t r = threadIdx.x; r < rows; r += blockDim.x) s += A[r * cols + c];
    red[threadIdx.x] = s;
    __syncthreads();
    for (int o = blockDim.x / 2; o > 0; o >>= 1) {
        if ((int)threadIdx.x < o) red[threadIdx.x] += red[threadIdx.x + o];
        __syncthreads();
    }
    if (threadIdx.x == 0) out[c] = red[0];
}

// dE rows from dX3: de_i = dx[:, 0:64] + dx[:, 128:192] sign(e_i - e_j),
//                   de_j = dx[:, 64:128] - dx[:, 128:192] sign(e_i - e_j)
__global__ void k_sur_split(const float* __restrict__ dX3, const float* __restrict__ E, int64_t B,
                            float* __restrict__ dE) {
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < B * kE;
         e += (int64_t)gridDim.x * blockDim.x) {
        const int64_t b = e / kE;
        const int q = (int)(e % kE);
        const float d = E[b * kE + q] - E[(B + b) * kE + q];
        const float sg = d > 0.f ? 1.f : (d < 0.f ? -1.f : 0.f);
        const float dd = dX3[b * kHeadIn + 2 * kE + q] * sg;
        dE[b * kE + q] = dX3[b * kHeadIn + q] + dd;
        dE[(B + b) * kE + q] = dX3[b * kHeadIn + kE + q] - dd;
    }
}

// One training step's values, read from device memory by the kernels of a
// step that is replayed from a CUDA graph (cursor = the step's index).
struct SurStep {
    int64_t start;  // first position of the batch in the epoch's order
    uint64_t step;  // the optimiser's step count before the step (swap stream)
    float c1, c2;   // Adam's bias corrections after the step
};

__global__ void k_sur_adam(float* __restrict__ w, const float* __restrict__ g, float* __restrict__ m,
                           float* __restrict__ v, int64_t P, float lr, float c1, float c2,
                           __nv_bfloat16* __restrict__ wb, PadW pw, const SurStep* __restrict__ sp,
                           const int* __restrict__ cursor) {
    if (sp) {
        c1 = sp[*cursor].c1;
        c2 = sp[*cursor].c2;
    }
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < P;
         i += (int64_t)gridDim.x * blockDim.x) {
        const float gi = g[i];
        const float mi = 0.9f * m[i] + 0.1f * gi;
        const float vi = 0.999f * v[i] + 0.001f * gi * gi;
        m[i] = mi;
        v[i] = vi;
        const float wi = w[i] - lr * (mi / c1) / (sqrtf(vi / c2) + 1e-8f);
        w[i] = wi;
        const __nv_bfloat16 h = __float2bfloat16_rn(wi);
        wb[i] = h;
        pad_store(pw, i, h);
    }
}

// o = o * a + b
__global__ void k_sur_affine(float* __restrict__ o, int64_t n, float a, float b) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x)
        o[i] = fmaf(o[i], a, b);
}

// rows of a [rows][cols] matrix += bias
__global__ void k_sur_add_bias(float* __restrict__ A, const float* __restrict__ bias, int64_t rows,
                               int cols) {
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < rows * cols;
         e += (int64_t)gridDim.x * blockDim.x)
        A[e] += bias[e % cols];
}

__global__ void k_sur_cast(const float* __restrict__ w, int64_t P, __nv_bfloat16* __restrict__ wb,
                           PadW pw) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < P;
         i += (int64_t)gridDim.x * blockDim.x) {
        const __nv_bfloat16 h = __float2bfloat16_rn(w[i]);
        wb[i] = h;
        pad_store(pw, i, h);
    }
}

// training batch: rows 0..B-1 = first points, B..2B-1 = second points; each
// pair is swapped with probability 1/2 (Philox block {step, b, 7, 0})
__global__ void k_sur_batch(const uint32_t* __restrict__ pa, const uint32_t* __restrict__ pb,
                            const float* __restrict__ tgt, const int64_t* __restrict__ order,
                            int64_t start, int64_t B, uint64_t seed, uint64_t step, int swap,
                            uint32_t* __restrict__ pts, float* __restrict__ tb,
                            const SurStep* __restrict__ sp = nullptr,
                            const int* __restrict__ cursor = nullptr) {
    if (sp) {
        start = sp[*cursor].start;
        step = sp[*cursor].step;
    }
    for (int64_t b = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; b < B;
         b += (int64_t)gridDim.x * blockDim.x) {
        const int64_t s = order ? order[start + b] : start + b;
        uint32_t x = pa[s], y = pb[s];
        if (swap) {
            uint64_t c[4] = {step, (uint64_t)b, 7, 0};
            philox4x64_10(c, seed, 0x5ee9ull);
            if (c[0] & 1) {
                const uint32_t tmp = x;
                x = y;
                y = tmp;
            }
        }
        pts[b] = x;
        pts[B + b] = y;
        tb[b] = tgt ? tgt[s] : 0.f;
    }
}

__global__ void k_sur_next(int* cursor) { *cursor += 1; }

// linear pair index a * nb + b -> point ids of the pair
__global__ void k_sur_ids_to_pairs(const uint32_t* __restrict__ ids, int64_t count,
                                   const uint32_t* __restrict__ pts_a,
                                   const uint32_t* __restrict__ pts_b, int64_t nb,
                                   uint32_t* __restrict__ pa, uint32_t* __restrict__ pb) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < count;
         i += (int64_t)gridDim.x * blockDim.x) {
        const uint32_t id = ids[i];
        pa[i] = pts_a[id / nb];
        pb[i] = pts_b[id % nb];
    }
}

}  // namespace cc

// ============================================================================
using namespace cc;

struct cc_sur {
    int n = 0;
    SurOff off{1};
    DevMem w, wb, g, m, v;
    DevMem wp;  // padded BF16 W1 and W3 (PadW)
    int64_t step = 0;
    float tmean = 0.f, tsd = 1.f;
    // batch scratch
    int64_t cap = 0;
    DevMem pts, tb, X0, A1, H1, Ef, E, X3, A3, H3, y, dy, dA3, dX3, dE, dH1, dA1, loss;
    DevMem order;
    DevMem ws;  // split-K partials of the weight-gradient GEMMs: w4 / b4 chunks,
    DevMem ws3, ws2, ws1;  // W3 / b3, W2 / b2, W1 / b1 (reduced together at the end)
    DevMem steps;  // per-step values of a training epoch, then the step cursor
};

namespace {

cc_status sfail(cc_ctx* c, cc_status s, const char* fmt, ...) {
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

#define SK(call)                                                                             \
    do {                                                                                     \
        cudaError_t _e = (call);                                                             \
        if (_e != cudaSuccess) {                                                             \
            cudaGetLastError();                                                              \
            return sfail(ctx, _e == cudaErrorMemoryAllocation ? CC_ERR_OOM : CC_ERR_CUDA,    \
                         "%s: %s", #call, cudaGetErrorString(_e));                           \
        }                                                                                    \
    } while (0)

unsigned grid1(int64_t n) {
    int64_t b = (n + 255) / 256;
    return (unsigned)std::max<int64_t>(1, std::min<int64_t>(b, (int64_t)sm_count() * 16));
}

cc_status ensure_batch(cc_ctx* ctx, cc_sur* s, int64_t B) {
    if (B <= s->cap) return CC_OK;
    const int n = s->n;
    SK(s->pts.alloc(8 * B));
    SK(s->tb.alloc(4 * B));
    SK(s->X0.alloc(2 * 2 * B * ldz(n)));
    SK(s->A1.alloc(4 * 2 * B * kH1));
    SK(s->H1.alloc(2 * 2 * B * kH1));
    SK(s->Ef.alloc(4 * 2 * B * kE));
    SK(s->E.alloc(4 * 2 * B * kE));
    SK(s->X3.alloc(2 * B * kHeadInP));
    SK(s->A3.alloc(4 * B * kH3));
    SK(s->H3.alloc(2 * B * kH3));
    SK(s->y.alloc(4 * B));
    SK(s->dy.alloc(4 * B));
    SK(s->dA3.alloc(4 * B * kH3));
    SK(s->dX3.alloc(4 * B * kHeadIn));
    SK(s->dE.alloc(4 * 2 * B * kE));
    SK(s->dH1.alloc(4 * 2 * B * kH1));
    SK(s->dA1.alloc(4 * 2 * B * kH1));
    SK(s->loss.alloc(8));
    s->cap = B;
    return CC_OK;
}

typedef __nv_bfloat16 bf16;

PadW padw(cc_sur* s) { return PadW{s->wp.as<bf16>(), s->off.W1, s->off.W3, s->n}; }
const bf16* w1p(cc_sur* s) { return s->wp.as<bf16>(); }
const bf16* w3p(cc_sur* s) { return s->wp.as<bf16>() + (int64_t)kH1 * ldz(s->n); }

// forward over a batch whose point list (2B entries) is in s->pts; with t,
// also the loss (sum of squares into s->loss) and dy
cc_status forward(cc_ctx* ctx, cc_sur* s, const Field& f, int64_t B, const float* t) {
    cudaStream_t st = ctx->stream;
    const int n = s->n;
    const SurOff& o = s->off;
    const bf16* wb = s->wb.as<bf16>();
    const float* w = s->w.as<float>();
    note_launch(5);
    k_sur_gather_z<<<grid1(2 * B * n), 256, 0, st>>>(f.zhat.as<float>(), n, f.n_pad,
                                                     sqrtf((float)(n - 1)), s->pts.as<uint32_t>(),
                                                     2 * B, ldz(n), s->X0.as<bf16>());
    SK(tmm(ctx->status.as<int>(), s->X0.as<bf16>(), ldz(n), 1, w1p(s), 1, ldz(n), s->A1.as<float>(),
           kH1, (int)(2 * B), kH1, n, st));
    k_sur_bias_gelu<<<grid1(2 * B * kH1), 256, 0, st>>>(s->A1.as<float>(), w + o.b1, 2 * B, kH1,
                                                        s->H1.as<bf16>());
    SK(tmm(ctx->status.as<int>(), s->H1.as<bf16>(), kH1, 1, wb + o.W2, 1, kH1, s->Ef.as<float>(), kE,
           (int)(2 * B), kE, kH1, st));
    const uint32_t* pts = s->pts.as<uint32_t>();
    k_sur_head_input<<<grid1(B * kHeadIn), 256, 0, st>>>(s->Ef.as<float>(), w + o.b2, pts,
                                                         pts + B, f.X, f.Y, f.Z, B,
                                                         s->X3.as<bf16>(), s->E.as<float>());
    SK(tmm(ctx->status.as<int>(), s->X3.as<bf16>(), kHeadInP, 1, w3p(s), 1, kHeadInP,
           s->A3.as<float>(), kH3, (int)B, kH3, kHeadIn, st));
    k_sur_bias_gelu<<<grid1(B * kH3), 256, 0, st>>>(s->A3.as<float>(), w + o.b3, B, kH3,
                                                    s->H3.as<bf16>());
    if (t) SK(cudaMemsetAsync(s->loss.p, 0, 8, st));
    // with targets, also the head's GELU backward dA3 = (dy w4) gelu'(A3)
    k_sur_out<<<grid1(B * 32), 256, 0, st>>>(s->H3.as<bf16>(), w + o.w4, w + o.b4, t, B, s->tmean,
                                             1.f / s->tsd, s->y.as<float>(), s->dy.as<float>(),
                                             s->loss.as<double>(), s->A3.as<float>(),
                                             s->dA3.as<float>());
    SK(cudaGetLastError());
    return CC_OK;
}

// gradients of the batch loss into s->g (overwritten)
cc_status backward(cc_ctx* ctx, cc_sur* s, int64_t B) {
    cudaStream_t st = ctx->stream;
    const int n = s->n;
    const SurOff& o = s->off;
    const bf16* wb = s->wb.as<bf16>();
    float* g = s->g.as<float>();
    // the weight gradients' partials are summed by one launch at the end
    ReduceSegs segs;
    // head output layer: w4 and b4 (adjacent) from per-chunk partial sums
    {
        const int64_t nb = (B + 63) / 64;
        SK(s->ws.ensure(sizeof(float) * (size_t)nb * (kH3 + 1)));
        note_launch();
        k_sur_w4_grad<<<(unsigned)nb, kH3 + 32, 0, st>>>(s->H3.as<bf16>(), s->dy.as<float>(), B,
                                                         s->ws.as<float>());
        segs.s[0] = ReduceSeg{s->ws.as<float>(), (int)nb, 1, kH3 + 1, g + o.w4, kH3 + 1, nullptr,
                              reduce_blocks(kH3 + 1)};
    }
    SK(tmm(ctx->status.as<int>(), s->dA3.as<float>(), 1, kH3, s->X3.as<bf16>(), kHeadInP, 1,
           g + o.W3, kHeadIn, kH3, kHeadIn, (int)B, st, &s->ws3, g + o.b3, &segs.s[1]));
    SK(tmm(ctx->status.as<int>(), s->dA3.as<float>(), kH3, 1, w3p(s), kHeadInP, 1,
           s->dX3.as<float>(), kHeadIn, (int)B, kHeadIn, kH3, st));
    k_sur_split<<<grid1(B * kE), 256, 0, st>>>(s->dX3.as<float>(), s->E.as<float>(), B,
                                               s->dE.as<float>());
    // encoder
    SK(tmm(ctx->status.as<int>(), s->dE.as<float>(), 1, kE, s->H1.as<bf16>(), kH1, 1, g + o.W2,
           kH1, kE, kH1, (int)(2 * B), st, &s->ws2, g + o.b2, &segs.s[2]));
    note_launch(2);
    SK(tmm(ctx->status.as<int>(), s->dE.as<float>(), kE, 1, wb + o.W2, kH1, 1, s->dH1.as<float>(),
           kH1, (int)(2 * B), kH1, kE, st));
    k_sur_gelu_bwd<<<grid1(2 * B * kH1), 256, 0, st>>>(s->A1.as<float>(), nullptr, nullptr,
                                                       s->dH1.as<float>(), 2 * B, kH1,
                                                       s->dA1.as<float>());
    SK(tmm(ctx->status.as<int>(), s->dA1.as<float>(), 1, kH1, s->X0.as<bf16>(), ldz(n), 1, g + o.W1,
           n, kH1, n, (int)(2 * B), st, &s->ws1, g + o.b1, &segs.s[3]));
    unsigned blocks = 0;
    for (const ReduceSeg& r : segs.s) blocks += r.blocks;
    if (blocks) {
        note_launch();
        k_mm_reduce_multi<<<blocks, 256, 0, st>>>(segs);
    }
    SK(cudaGetLastError());
    return CC_OK;
}

Field* sfield(cc_ctx* ctx, int32_t id) {
    if (id < 0 || id >= (int32_t)ctx->fields.size()) return nullptr;
    return ctx->fields[id].get();
}

// device status word after a screen (the tensor-core kernel's bounded waits)
cc_status screen_status(cc_ctx* ctx) {
    int st = 0;
    SK(cudaMemcpyAsync(&st, ctx->status.p, sizeof(int), cudaMemcpyDeviceToHost, ctx->stream));
    SK(cudaStreamSynchronize(ctx->stream));
    if (st == DEV_OK) return CC_OK;
    SK(cudaMemsetAsync(ctx->status.p, 0, sizeof(int), ctx->stream));
    return sfail(ctx, st == DEV_TIMEOUT ? CC_ERR_TIMEOUT : CC_ERR_CUDA,
                 "surrogate screen: device status %d", st);
}

// Predictions for every pair of two regions of one field into pred [|A|][|B|]
// (self region pairs: -inf for b <= a).
cc_status screen_predict(cc_ctx* ctx, cc_sur* s, int32_t region_a, int32_t region_b,
                         DevMem& pred, Region** ra_out, Region** rb_out) {
    if (region_a < 0 || region_a >= (int)ctx->regions.size() || !ctx->regions[region_a] ||
        region_b < 0 || region_b >= (int)ctx->regions.size() || !ctx->regions[region_b])
        return sfail(ctx, CC_ERR_INVALID_ARG, "unknown region");
    Region& ra = *ctx->regions[region_a];
    Region& rb = *ctx->regions[region_b];
    if (ra.field != rb.field) return sfail(ctx, CC_ERR_INVALID_ARG, "regions of one field only");
    Field* f = sfield(ctx, ra.field);
    if (!f || f->n != s->n) return sfail(ctx, CC_ERR_INVALID_ARG, "field does not match");
    if ((uint64_t)ra.np * rb.np >= (1ull << 32))
        return sfail(ctx, CC_ERR_INVALID_ARG, "|A| * |B| must be below 2^32");
    cudaStream_t st = ctx->stream;
    const int n = s->n;
    const SurOff& o = s->off;
    const int64_t na = ra.np, nb = rb.np;
    cc_status r = ensure_batch(ctx, s, (std::max(na, nb) + 1) / 2);
    if (r) return r;
    DevMem Ea, Eb, Ua;
    SK(Ea.alloc(4 * na * kE));
    SK(Eb.alloc(4 * nb * kE));
    SK(Ua.alloc(4 * na * kH3));
    SK(pred.alloc(4 * (size_t)na * nb));
    const float* w = s->w.as<float>();
    // per-point encoder (bf16 weights, as in training) and head projections
    for (int side = 0; side < 2; ++side) {
        const Region& rg = side ? rb : ra;
        const int64_t np = rg.np;
        float* E = side ? Eb.as<float>() : Ea.as<float>();
        note_launch(2);
        k_sur_gather_z<<<grid1(np * n), 256, 0, st>>>(f->zhat.as<float>(), n, f->n_pad,
                                                      sqrtf((float)(n - 1)),
                                                      rg.pts.as<uint32_t>(), np, ldz(n),
                                                      s->X0.as<bf16>());
        SK(mm(s->X0.as<bf16>(), ldz(n), 1, s->wb.as<bf16>() + o.W1, 1, n, s->A1.as<float>(), kH1,
              (int)np, kH1, n, 0, st));
        k_sur_bias_gelu<<<grid1(np * kH1), 256, 0, st>>>(s->A1.as<float>(), w + o.b1, np, kH1,
                                                         s->H1.as<bf16>());
        SK(mm(s->H1.as<bf16>(), kH1, 1, s->wb.as<bf16>() + o.W2, 1, kH1, E, kE, (int)np, kE, kH1,
              0, st));
        note_launch();
        k_sur_add_bias<<<grid1(np * kE), 256, 0, st>>>(E, w + o.b2, np, kE);
        if (!side) {  // Wa e_a + b3 per point of A (Wb e_b is part of the contraction)
            SK(mm(E, kE, 1, w + o.W3, 1, kHeadIn, Ua.as<float>(), kH3, (int)np, kH3, kE, 0, st));
            note_launch();
            k_sur_add_bias<<<grid1(np * kH3), 256, 0, st>>>(Ua.as<float>(), w + o.b3, np, kH3);
        }
    }
    SK(launch_sur_screen_tc(Ea.as<float>(), Ua.as<float>(), Eb.as<float>(), s->wb.p, w, o.W3,
                            o.w4, o.b4, ra.pts.as<uint32_t>(), rb.pts.as<uint32_t>(), na, nb,
                            region_a == region_b, f->X, f->Y, f->Z, s->tmean, s->tsd,
                            pred.as<float>(), ctx->status.as<int>(), st));
    cc_status sr = screen_status(ctx);
    if (sr) return sr;
    SK(cudaGetLastError());
    *ra_out = &ra;
    *rb_out = &rb;
    return CC_OK;
}

}  // namespace

extern "C" {

cc_status cc_sur_create(cc_ctx* ctx, int n_members, uint64_t seed, cc_sur** out) {
    if (!ctx || !out || n_members < 2 || n_members > 1024)
        return sfail(ctx, CC_ERR_INVALID_ARG, "bad arguments");
    cc_sur* s = new (std::nothrow) cc_sur();
    if (!s) return CC_ERR_OOM;
    std::unique_ptr<cc_sur> guard(s);
    s->n = n_members;
    s->off = SurOff(n_members);
    const int64_t P = s->off.total;
    SK(s->w.alloc(4 * P));
    SK(s->wb.alloc(2 * P));
    SK(s->wp.alloc(2 * ((size_t)kH1 * ldz(n_members) + (size_t)kH3 * kHeadInP)));
    SK(cudaMemsetAsync(s->wp.p, 0, s->wp.bytes, ctx->stream));
    SK(s->g.alloc(4 * P));
    SK(s->m.alloc(4 * P));
    SK(s->v.alloc(4 * P));
    // seeded init: weights ~ N(0, 1 / fan_in) from Philox + Box-Muller, biases 0
    std::vector<float> h(P, 0.f);
    auto fill = [&](int64_t o, int rows, int cols, uint64_t tag) {
        for (int64_t i = 0; i < (int64_t)rows * cols; ++i) {
            uint64_t x = seed * 0x9E3779B97F4A7C15ull + tag * 0xD1B54A32D192ED03ull + (uint64_t)i;
            x ^= x >> 30;
            x *= 0xBF58476D1CE4E5B9ull;
            x ^= x >> 27;
            x *= 0x94D049BB133111EBull;
            x ^= x >> 31;
            const double u1 = ((double)(x >> 11) + 0.5) / 9007199254740992.0;
            x = x * 0x2545F4914F6CDD1Dull + 1;
            const double u2 = ((double)(x >> 11) + 0.5) / 9007199254740992.0;
            h[o + i] = (float)(sqrt(-2.0 * log(u1)) * cos(6.283185307179586 * u2) / sqrt((double)cols));
        }
    };
    fill(s->off.W1, kH1, n_members, 1);
    fill(s->off.W2, kE, kH1, 2);
    fill(s->off.W3, kH3, kHeadIn, 3);
    fill(s->off.w4, 1, kH3, 4);
    cc_status st = cc_sur_set_params(ctx, s, h.data());
    if (st) return st;
    *out = guard.release();
    return CC_OK;
}

cc_status cc_sur_set_params(cc_ctx* ctx, cc_sur* s, const float* params) {
    if (!ctx || !s || !params) return CC_ERR_INVALID_ARG;
    const int64_t P = s->off.total;
    SK(cudaMemcpyAsync(s->w.p, params, 4 * P, cudaMemcpyHostToDevice, ctx->stream));
    SK(cudaMemsetAsync(s->m.p, 0, 4 * P, ctx->stream));
    SK(cudaMemsetAsync(s->v.p, 0, 4 * P, ctx->stream));
    note_launch();
    k_sur_cast<<<grid1(P), 256, 0, ctx->stream>>>(s->w.as<float>(), P, s->wb.as<bf16>(),
                                                  padw(s));
    SK(cudaGetLastError());
    SK(cudaStreamSynchronize(ctx->stream));
    s->step = 0;
    return CC_OK;
}

cc_status cc_sur_get_params(cc_ctx* ctx, cc_sur* s, float* params, int64_t* n_params,
                            float* target_mean, float* target_sd) {
    if (!ctx || !s) return CC_ERR_INVALID_ARG;
    if (n_params) *n_params = s->off.total;
    if (target_mean) *target_mean = s->tmean;
    if (target_sd) *target_sd = s->tsd;
    if (params) {
        SK(cudaMemcpyAsync(params, s->w.p, 4 * s->off.total, cudaMemcpyDeviceToHost, ctx->stream));
        SK(cudaStreamSynchronize(ctx->stream));
    }
    return CC_OK;
}

cc_status cc_sur_set_target_scale(cc_ctx* ctx, cc_sur* s, float mean, float sd) {
    if (!ctx || !s || !(sd > 0.f)) return sfail(ctx, CC_ERR_INVALID_ARG, "sd must be > 0");
    s->tmean = mean;
    s->tsd = sd;
    return CC_OK;
}

cc_status cc_sur_loss_grad(cc_ctx* ctx, cc_sur* s, int32_t field_id, const uint32_t* pa,
                           const uint32_t* pb, const float* target, int64_t n_pairs, float* loss,
                           float* grad) {
    if (!ctx || !s || !pa || !pb || !target || n_pairs < 1)
        return sfail(ctx, CC_ERR_INVALID_ARG, "bad arguments");
    Field* f = sfield(ctx, field_id);
    if (!f || f->n != s->n) return sfail(ctx, CC_ERR_INVALID_ARG, "field does not match");
    cc_status st = ensure_batch(ctx, s, n_pairs);
    if (st) return st;
    std::vector<uint32_t> pts(2 * n_pairs);
    for (int64_t i = 0; i < n_pairs; ++i) {
        if (pa[i] >= (uint64_t)f->P || pb[i] >= (uint64_t)f->P)
            return sfail(ctx, CC_ERR_INVALID_ARG, "point id out of range");
        pts[i] = pa[i];
        pts[n_pairs + i] = pb[i];
    }
    SK(cudaMemcpyAsync(s->pts.p, pts.data(), 8 * n_pairs, cudaMemcpyHostToDevice, ctx->stream));
    SK(cudaMemcpyAsync(s->tb.p, target, 4 * n_pairs, cudaMemcpyHostToDevice, ctx->stream));
    if ((st = forward(ctx, s, *f, n_pairs, s->tb.as<float>()))) return st;
    if ((st = backward(ctx, s, n_pairs))) return st;
    double l = 0;
    SK(cudaMemcpyAsync(&l, s->loss.p, 8, cudaMemcpyDeviceToHost, ctx->stream));
    if (grad)
        SK(cudaMemcpyAsync(grad, s->g.p, 4 * s->off.total, cudaMemcpyDeviceToHost, ctx->stream));
    SK(cudaStreamSynchronize(ctx->stream));
    if (loss) *loss = (float)(l / n_pairs);
    return CC_OK;
}

cc_status cc_sur_train(cc_ctx* ctx, cc_sur* s, int32_t field_id, const uint32_t* pa,
                       const uint32_t* pb, const float* target, int64_t n_pairs, int on_device,
                       int epochs, int batch, float lr, uint64_t seed, float* epoch_loss) {
    if (!ctx || !s || !pa || !pb || !target || n_pairs < 1 || epochs < 0 || batch < 1 ||
        !(lr > 0.f))
        return sfail(ctx, CC_ERR_INVALID_ARG, "bad arguments");
    Field* f = sfield(ctx, field_id);
    if (!f || f->n != s->n) return sfail(ctx, CC_ERR_INVALID_ARG, "field does not match");
    cudaStream_t st = ctx->stream;
    const uint32_t *da = pa, *db = pb;
    const float* dt = target;
    DevMem ha, hb, ht;
    if (!on_device) {
        SK(ha.alloc(4 * n_pairs));
        SK(hb.alloc(4 * n_pairs));
        SK(ht.alloc(4 * n_pairs));
        SK(cudaMemcpyAsync(ha.p, pa, 4 * n_pairs, cudaMemcpyHostToDevice, st));
        SK(cudaMemcpyAsync(hb.p, pb, 4 * n_pairs, cudaMemcpyHostToDevice, st));
        SK(cudaMemcpyAsync(ht.p, target, 4 * n_pairs, cudaMemcpyHostToDevice, st));
        da = ha.as<uint32_t>();
        db = hb.as<uint32_t>();
        dt = ht.as<float>();
    }
    const int64_t B = std::min<int64_t>(batch, n_pairs);
    const int64_t steps = n_pairs / B;
    // per-epoch shuffle: a seeded permutation (host Fisher-Yates on SplitMix64).
    // Epoch e + 1's permutation is built by a second host thread into the
    // other of two pinned buffers while epoch e's steps run on the GPU (the
    // generator is used by one thread at a time, in epoch order, so every
    // permutation is the one a sequential loop would draw); an event per
    // buffer marks when its copy to the device has been done.
    SK(s->order.ensure(8 * n_pairs));
    HostMem* order_h = ctx->sur_order;  // pinned, kept by the context for later calls
    SK(order_h[0].ensure(8 * n_pairs));
    SK(order_h[1].ensure(8 * n_pairs));
    uint64_t rs = seed ^ 0xA0761D6478BD642Full;
    auto next = [&]() {
        rs += 0x9E3779B97F4A7C15ull;
        uint64_t z = rs;
        z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
        z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
        return z ^ (z >> 31);
    };
    auto shuffle_into = [&](int64_t* order) {
        for (int64_t i = 0; i < n_pairs; ++i) order[i] = i;
        for (int64_t i = n_pairs - 1; i > 0; --i) std::swap(order[i], order[next() % (i + 1)]);
    };
    struct Worker {  // joined on every way out of this function
        std::thread t;
        void join() {
            if (t.joinable()) t.join();
        }
        ~Worker() { join(); }
    } worker;
    struct Events {
        cudaEvent_t e[2] = {nullptr, nullptr};
        bool used[2] = {false, false};
        ~Events() {
            for (cudaEvent_t x : e)
                if (x) cudaEventDestroy(x);
        }
    } copied;
    for (int b = 0; b < 2; ++b)
        SK(cudaEventCreateWithFlags(&copied.e[b], cudaEventDisableTiming));
    // loss reads every 64 steps land in pinned memory without a host wait
    const int64_t reads = (steps + 63) / 64;
    SK(ctx->sur_loss.ensure(sizeof(double) * (size_t)std::max<int64_t>(1, reads * epochs)));
    double* loss_h = ctx->sur_loss.as<double>();
    // the first permutation is drawn while the targets are standardized
    if (epochs > 0) worker.t = std::thread(shuffle_into, order_h[0].as<int64_t>());
    // target standardization from the training targets
    {
        std::vector<float> h(n_pairs);
        SK(cudaMemcpyAsync(h.data(), dt, 4 * n_pairs, cudaMemcpyDeviceToHost, st));
        SK(cudaStreamSynchronize(st));
        double m = 0, v = 0;
        for (float x : h) m += x;
        m /= n_pairs;
        for (float x : h) v += (x - m) * (x - m);
        v /= n_pairs;
        s->tmean = (float)m;
        s->tsd = (float)std::max(sqrt(v), 1e-6);
    }
    cc_status r = ensure_batch(ctx, s, B);
    if (r) return r;
    // Each step's kernels read the step's batch offset, swap stream and Adam
    // corrections from a device table (one entry per step of the epoch); the
    // first step runs directly, the second is captured into a CUDA graph
    // (every buffer is sized by then) and the graph is replayed for the rest,
    // so the GPU runs a step's ~25 launches back to back.
    SK(s->steps.ensure(sizeof(SurStep) * (size_t)steps + 16));
    SurStep* dsteps = s->steps.as<SurStep>();
    int* cursor = reinterpret_cast<int*>(dsteps + steps);
    std::vector<SurStep> hsteps((size_t)steps);
    cudaGraphExec_t exec = nullptr;
    int graph_kernels = 0;
    auto body = [&]() -> cc_status {
        cc_status r2;
        note_launch();
        k_sur_batch<<<grid1(B), 256, 0, st>>>(da, db, dt, s->order.as<int64_t>(), 0, B, seed, 0,
                                              1, s->pts.as<uint32_t>(), s->tb.as<float>(), dsteps,
                                              cursor);
        if ((r2 = forward(ctx, s, *f, B, s->tb.as<float>()))) return r2;
        if ((r2 = backward(ctx, s, B))) return r2;
        note_launch(2);
        k_sur_adam<<<grid1(s->off.total), 256, 0, st>>>(s->w.as<float>(), s->g.as<float>(),
                                                        s->m.as<float>(), s->v.as<float>(),
                                                        s->off.total, lr, 1.f, 1.f,
                                                        s->wb.as<bf16>(), padw(s), dsteps, cursor);
        k_sur_next<<<1, 1, 0, st>>>(cursor);
        SK(cudaGetLastError());
        return CC_OK;
    };
    cc_status res = CC_OK;
    for (int ep = 0; ep < epochs && res == CC_OK; ++ep) {
        const int b = ep & 1;
        worker.join();  // this epoch's permutation is complete
        SK(cudaMemcpyAsync(s->order.p, order_h[b].p, 8 * n_pairs, cudaMemcpyHostToDevice, st));
        SK(cudaEventRecord(copied.e[b], st));
        copied.used[b] = true;
        if (ep + 1 < epochs) {  // the next one, into the other buffer once its copy is done
            if (copied.used[b ^ 1]) SK(cudaEventSynchronize(copied.e[b ^ 1]));
            worker.t = std::thread(shuffle_into, order_h[b ^ 1].as<int64_t>());
        }
        for (int64_t k = 0; k < steps; ++k) {
            const int64_t t = s->step + k + 1;
            hsteps[k] = SurStep{k * B, (uint64_t)(s->step + k), 1.f - powf(0.9f, (float)t),
                                1.f - powf(0.999f, (float)t)};
        }
        SK(cudaMemcpyAsync(dsteps, hsteps.data(), sizeof(SurStep) * (size_t)steps,
                           cudaMemcpyHostToDevice, st));
        SK(cudaMemsetAsync(cursor, 0, sizeof(int), st));
        for (int64_t k = 0; k < steps; ++k) {
            if (exec) {
                note_launch(graph_kernels);
                SK(cudaGraphLaunch(exec, st));
            } else if (k == 0 || steps < 3) {
                if ((res = body())) break;
            } else {
                uint64_t before = 0, after = 0;
                cc_launch_count(&before);
                SK(cudaStreamBeginCapture(st, cudaStreamCaptureModeRelaxed));
                const cc_status rb = body();
                cudaGraph_t g = nullptr;
                const cudaError_t ec = cudaStreamEndCapture(st, &g);
                cc_launch_count(&after);
                graph_kernels = (int)(after - before);
                note_launch(-graph_kernels);
                if (rb != CC_OK || ec != cudaSuccess) {
                    if (g) cudaGraphDestroy(g);
                    cudaGetLastError();
                    res = rb != CC_OK ? rb : sfail(ctx, CC_ERR_CUDA, "step capture: %s",
                                                   cudaGetErrorString(ec));
                    break;
                }
                const cudaError_t ei = cudaGraphInstantiate(&exec, g, 0);
                cudaGraphDestroy(g);
                SK(ei);
                note_launch(graph_kernels);
                SK(cudaGraphLaunch(exec, st));
            }
            if (epoch_loss && (k % 64 == 63 || k == steps - 1))  // read k / 64 of the epoch
                SK(cudaMemcpyAsync(loss_h + ep * reads + k / 64, s->loss.p, 8,
                                   cudaMemcpyDeviceToHost, st));
        }
        s->step += steps;
    }
    if (exec) cudaGraphExecDestroy(exec);
    if (res) return res;
    SK(cudaStreamSynchronize(st));
    if (epoch_loss) {  // the mean of each epoch's loss reads, in read order
        for (int ep = 0; ep < epochs; ++ep) {
            double sum = 0;
            for (int64_t j = 0; j < reads; ++j) sum += loss_h[ep * reads + j] / B;
            epoch_loss[ep] = (float)(sum / reads);
        }
    }
    return CC_OK;
}

cc_status cc_sur_predict(cc_ctx* ctx, cc_sur* s, int32_t field_id, const uint32_t* pa,
                         const uint32_t* pb, int64_t n_pairs, int pairs_on_device, float* out,
                         int out_on_device) {
    if (!ctx || !s || !pa || !pb || !out || n_pairs < 0)
        return sfail(ctx, CC_ERR_INVALID_ARG, "bad arguments");
    Field* f = sfield(ctx, field_id);
    if (!f || f->n != s->n) return sfail(ctx, CC_ERR_INVALID_ARG, "field does not match");
    cudaStream_t st = ctx->stream;
    const int64_t B = std::min<int64_t>(n_pairs, 1 << 16);
    cc_status r = ensure_batch(ctx, s, std::max<int64_t>(B, 1));
    if (r) return r;
    DevMem hpa, hpb, hout;
    const uint32_t *da = pa, *db = pb;
    float* dout = out;
    if (!pairs_on_device) {
        SK(hpa.alloc(4 * std::max<int64_t>(n_pairs, 1)));
        SK(hpb.alloc(4 * std::max<int64_t>(n_pairs, 1)));
        SK(cudaMemcpyAsync(hpa.p, pa, 4 * n_pairs, cudaMemcpyHostToDevice, st));
        SK(cudaMemcpyAsync(hpb.p, pb, 4 * n_pairs, cudaMemcpyHostToDevice, st));
        da = hpa.as<uint32_t>();
        db = hpb.as<uint32_t>();
    }
    if (!out_on_device) {
        SK(hout.alloc(4 * std::max<int64_t>(n_pairs, 1)));
        dout = hout.as<float>();
    }
    for (int64_t s0 = 0; s0 < n_pairs; s0 += B) {
        const int64_t b = std::min(B, n_pairs - s0);
        note_launch();
        k_sur_batch<<<grid1(b), 256, 0, st>>>(da, db, nullptr, nullptr, s0, b, 0, 0, 0,
                                              s->pts.as<uint32_t>(), s->tb.as<float>());
        if ((r = forward(ctx, s, *f, b, nullptr))) return r;
        // de-standardize y into the output
        SK(cudaMemcpyAsync(dout + s0, s->y.p, 4 * b, cudaMemcpyDeviceToDevice, st));
    }
    // outputs hold standardized predictions: back to the target's units
    note_launch();
    k_sur_affine<<<grid1(n_pairs), 256, 0, st>>>(dout, n_pairs, s->tsd, s->tmean);
    SK(cudaGetLastError());
    if (!out_on_device) {
        SK(cudaMemcpyAsync(out, dout, 4 * n_pairs, cudaMemcpyDeviceToHost, st));
        SK(cudaStreamSynchronize(st));
    }
    return CC_OK;
}

cc_status cc_sur_screen(cc_ctx* ctx, cc_sur* s, int32_t region_a, int32_t region_b, int topk,
                        uint64_t* ids, float* preds) {
    if (!ctx || !s || topk < 1 || topk > 8192 || !ids || !preds)
        return sfail(ctx, CC_ERR_INVALID_ARG, "bad arguments (1 <= topk <= 8192)");
    DevMem pred, aux;
    Region *pra = nullptr, *prb = nullptr;
    cc_status r = screen_predict(ctx, s, region_a, region_b, pred, &pra, &prb);
    if (r) return r;
    cudaStream_t st = ctx->stream;
    const int64_t na = pra->np, nb = prb->np;
    // top-k by histogram selection, then one sorting CTA
    const size_t o_hist = 0, o_sel = 4 * 4096, o_idx = o_sel + 256, o_tv = o_idx + 4 * 8192,
                 o_ti = o_tv + 4 * 8192, o_sk = o_ti + 8 * 8192;
    SK(aux.alloc(o_sk + 8 * 8192));
    unsigned char* ab = aux.as<unsigned char>();
    SK(cudaMemsetAsync(ab, 0, o_idx, st));
    const int64_t N = na * nb;
    SK(launch_select_top(pred.as<float>(), N, 1.f, (unsigned)topk, (unsigned*)(ab + o_hist),
                         (Select*)(ab + o_sel), (uint32_t*)(ab + o_idx), 8192, st));
    // candidate indices are the linear pair indices a * nb + b themselves
    SK(launch_sort_top_ids(pred.as<float>(), (const uint32_t*)(ab + o_idx),
                           &((Select*)(ab + o_sel))->count, 8192, topk, (float*)(ab + o_tv),
                           (unsigned long long*)(ab + o_ti), (unsigned long long*)(ab + o_sk),
                           st));
    SK(cudaMemcpyAsync(preds, ab + o_tv, 4 * (size_t)topk, cudaMemcpyDeviceToHost, st));
    SK(cudaMemcpyAsync(ids, ab + o_ti, 8 * (size_t)topk, cudaMemcpyDeviceToHost, st));
    SK(cudaStreamSynchronize(st));
    return CC_OK;
}

cc_status cc_sur_screen_verify(cc_ctx* ctx, cc_sur* s, int32_t region_a, int32_t region_b,
                               int64_t budget, const cc_params* params, cc_rp_result* out) {
    if (!ctx || !s || !params || !out || budget < 1 || budget > (1 << 24))
        return sfail(ctx, CC_ERR_INVALID_ARG, "bad arguments (1 <= budget <= 2^24)");
    DevMem pred, aux, pairs;
    Region *pra = nullptr, *prb = nullptr;
    cc_status r = screen_predict(ctx, s, region_a, region_b, pred, &pra, &prb);
    if (r) return r;
    cudaStream_t st = ctx->stream;
    const int64_t na = pra->np, nb = prb->np, N = na * nb;
    // the budget's largest predictions (threshold selection; ties at the cut
    // fill up to a quarter more before the rest is dropped)
    const int64_t cap = std::min<int64_t>(N, budget + std::max<int64_t>(budget / 4, 4096));
    const size_t o_hist = 0, o_sel = 4 * 4096, o_idx = o_sel + 256;
    SK(aux.alloc(o_idx + 4 * (size_t)cap));
    unsigned char* ab = aux.as<unsigned char>();
    SK(cudaMemsetAsync(ab, 0, o_idx, st));
    uint32_t* idx = (uint32_t*)(ab + o_idx);
    SK(launch_select_top(pred.as<float>(), N, 1.f, (unsigned)budget, (unsigned*)(ab + o_hist),
                         (Select*)(ab + o_sel), idx, (unsigned)cap, st));
    Select hs;
    SK(cudaMemcpyAsync(&hs, ab + o_sel, sizeof hs, cudaMemcpyDeviceToHost, st));
    SK(cudaStreamSynchronize(st));
    const int64_t cnt = std::min<int64_t>(hs.count, cap);
    if (cnt == 0) {
        *out = cc_rp_result{-INFINITY, INFINITY, ~0ull, ~0ull, 0};
        return CC_OK;
    }
    SK(pairs.alloc(8 * (size_t)cnt));
    uint32_t* pa = pairs.as<uint32_t>();
    uint32_t* pb = pa + cnt;
    note_launch();
    k_sur_ids_to_pairs<<<grid1(cnt), 256, 0, st>>>(idx, cnt, pra->pts.as<uint32_t>(),
                                                   prb->pts.as<uint32_t>(), nb, pa, pb);
    SK(cudaGetLastError());
    const int64_t offs[2] = {0, cnt};
    r = cc_segment_extremes(ctx, pra->field, params, pa, pb, 1, offs, 1, nullptr, out);
    if (r) return r;
    // list positions -> linear pair indices of the region pair
    uint32_t lin[2] = {0, 0};
    if (out->argmax < (uint64_t)cnt)
        SK(cudaMemcpyAsync(&lin[0], idx + out->argmax, 4, cudaMemcpyDeviceToHost, st));
    if (out->argmin < (uint64_t)cnt)
        SK(cudaMemcpyAsync(&lin[1], idx + out->argmin, 4, cudaMemcpyDeviceToHost, st));
    SK(cudaStreamSynchronize(st));
    if (out->argmax < (uint64_t)cnt) out->argmax = lin[0];
    if (out->argmin < (uint64_t)cnt) out->argmin = lin[1];
    return CC_OK;
}

cc_status cc_sur_destroy(cc_ctx* ctx, cc_sur* s) {
    if (!s) return CC_ERR_INVALID_ARG;
    if (ctx) cudaStreamSynchronize(ctx->stream);
    delete s;
    return CC_OK;
}

}  // extern "C"
