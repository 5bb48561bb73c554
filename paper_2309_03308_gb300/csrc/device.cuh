// Device-side helpers shared by the kernels.
#pragma once

#include <cuda_runtime.h>
#include <math_constants.h>
#include <stdint.h>

namespace cc {

__device__ __forceinline__ void set_status(int* status, int code) {
    if (status) atomicCAS(status, 0, code);
}

__device__ __forceinline__ double warp_sum_f64(double v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// Knuth's TwoSum: s = fl(a + b) and the exact rounding error e (a + b = s + e)
// Packed fp32 pairs (lo, hi) in one 64-bit register, for the packed FMA
// fma.rn.f32x2: two independent IEEE fp32 fma.rn in one instruction.
__device__ __forceinline__ unsigned long long pack2(float lo, float hi) {
    unsigned long long r;
    asm("mov.b64 %0, {%1, %2};" : "=l"(r) : "f"(lo), "f"(hi));
    return r;
}
__device__ __forceinline__ void unpack2(unsigned long long v, float& lo, float& hi) {
    asm("mov.b64 {%0, %1}, %2;" : "=f"(lo), "=f"(hi) : "l"(v));
}
// d = a * b + d elementwise
__device__ __forceinline__ void ffma2(unsigned long long& d, unsigned long long a,
                                      unsigned long long b) {
    asm("fma.rn.f32x2 %0, %1, %2, %0;" : "+l"(d) : "l"(a), "l"(b));
}

__device__ __forceinline__ void two_sum(float a, float b, float& s, float& e) {
    s = __fadd_rn(a, b);
    const float bb = __fsub_rn(s, a);
    e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
}

// float-float accumulation (ah, al) += (bh, bl): TwoSum of the leading parts,
// low parts added, renormalised so |al| <= ulp(ah) / 2. Symmetric in its
// operands, so a butterfly reduction leaves every lane with the same value.
__device__ __forceinline__ void ff_add(float& ah, float& al, float bh, float bl) {
    float s, e;
    two_sum(ah, bh, s, e);
    e = __fadd_rn(e, __fadd_rn(al, bl));
    two_sum(s, e, ah, al);
}

__device__ __forceinline__ void warp_sum_ff(float& h, float& l) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        const float oh = __shfl_xor_sync(0xffffffffu, h, o);
        const float ol = __shfl_xor_sync(0xffffffffu, l, o);
        ff_add(h, l, oh, ol);
    }
}

__device__ __forceinline__ long long warp_sum_i64(long long v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// Warp sum of non-negative 64-bit values below 2^58 (each lane's value):
// three 32-bit reductions (redux.sync) of the high word and the two 16-bit
// halves of the low word, none of which can overflow over 32 lanes. Every
// lane receives the sum.
__device__ __forceinline__ long long warp_sum_u64_redux(long long v) {
    const unsigned long long u = (unsigned long long)v;
    const unsigned hi = __reduce_add_sync(0xffffffffu, (unsigned)(u >> 32));
    const unsigned mid = __reduce_add_sync(0xffffffffu, (unsigned)(u >> 16) & 0xffffu);
    const unsigned lo = __reduce_add_sync(0xffffffffu, (unsigned)u & 0xffffu);
    return (long long)(((unsigned long long)hi << 32) + ((unsigned long long)mid << 16) + lo);
}

__device__ __forceinline__ float warp_sum_f32(float v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// Philox4x64-10 (Salmon, Moraes, Dror, Shaw, SC 2011) from its published
// definition: 10 rounds of two 64x64->128 multiplies with the Weyl key
// schedule. c: counter in, output block out.
__device__ __forceinline__ void philox4x64_10(uint64_t c[4], uint64_t k0, uint64_t k1) {
#pragma unroll
    for (int r = 0; r < 10; ++r) {
        const uint64_t lo0 = 0xD2E7470EE14C6C93ull * c[0];
        const uint64_t hi0 = __umul64hi(0xD2E7470EE14C6C93ull, c[0]);
        const uint64_t lo1 = 0xCA5A826395121157ull * c[2];
        const uint64_t hi1 = __umul64hi(0xCA5A826395121157ull, c[2]);
        const uint64_t n0 = hi1 ^ c[1] ^ k0, n2 = hi0 ^ c[3] ^ k1;
        c[0] = n0;
        c[1] = lo1;
        c[2] = n2;
        c[3] = lo0;
        k0 += 0x9E3779B97F4A7C15ull;
        k1 += 0xBB67AE8584CAA73Bull;
    }
}

// Uniform [0, 1) with 24 random bits (exact in fp32): top 24 bits of a word.
__device__ __forceinline__ float u24(uint64_t w) {
    return (float)(unsigned)(w >> 40) * 5.9604644775390625e-8f;
}

// (value, index) extremes with the smallest index winning ties.
struct Ext {
    float vmax, vmin;
    unsigned long long imax, imin, count;
};

__device__ __forceinline__ Ext ext_empty() {
    Ext e;
    e.vmax = -CUDART_INF_F;
    e.vmin = CUDART_INF_F;
    e.imax = ~0ull;
    e.imin = ~0ull;
    e.count = 0;
    return e;
}

__device__ __forceinline__ void ext_add(Ext& e, float v, unsigned long long idx) {
    if (v > e.vmax || (v == e.vmax && idx < e.imax)) {
        e.vmax = v;
        e.imax = idx;
    }
    if (v < e.vmin || (v == e.vmin && idx < e.imin)) {
        e.vmin = v;
        e.imin = idx;
    }
    e.count++;
}

__device__ __forceinline__ void ext_merge(Ext& e, float vmax, unsigned long long imax, float vmin,
                                          unsigned long long imin, unsigned long long count) {
    if (vmax > e.vmax || (vmax == e.vmax && imax < e.imax)) {
        e.vmax = vmax;
        e.imax = imax;
    }
    if (vmin < e.vmin || (vmin == e.vmin && imin < e.imin)) {
        e.vmin = vmin;
        e.imin = imin;
    }
    e.count += count;
}

__device__ __forceinline__ Ext warp_ext(Ext e) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        float vmax = __shfl_xor_sync(0xffffffffu, e.vmax, o);
        float vmin = __shfl_xor_sync(0xffffffffu, e.vmin, o);
        unsigned long long imax = __shfl_xor_sync(0xffffffffu, e.imax, o);
        unsigned long long imin = __shfl_xor_sync(0xffffffffu, e.imin, o);
        unsigned long long c = __shfl_xor_sync(0xffffffffu, e.count, o);
        ext_merge(e, vmax, imax, vmin, imin, c);
    }
    return e;
}

}  // namespace cc
