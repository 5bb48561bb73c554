// Device building blocks of the KSG estimator (Section 3.2), shared by the
// pair-batch kernel (ksg.cu) and the batched sampling round (bos.cu).
//
// A pair (p, q) is staged by one warp into a shared-memory slot:
//   XO[t] = (x, y) of the sample at x-sorted position t (x ascending)
//   YO[u] = (y, x) of the sample at y-sorted position u (y ascending)
//   upos[t] = y-sorted position of the sample at x-sorted position t
// and each lane then evaluates whole samples with ksg_sample().
#pragma once

#include "device.cuh"

namespace cc {

// KMAX >= k: the list holds KMAX - k copies of -inf below the k real entries,
// so its last entry is always the k-th smallest seen.
template <int KMAX>
__device__ __forceinline__ void topk_insert(float (&top)[KMAX], float d) {
#pragma unroll
    for (int m = KMAX - 1; m > 0; --m) top[m] = fminf(top[m], fmaxf(top[m - 1], d));
    top[0] = fminf(top[0], d);
}

// ascending odd-even transposition sort of a register array
template <int KMAX>
__device__ __forceinline__ void sort_net(float (&t)[KMAX]) {
#pragma unroll
    for (int r = 0; r < KMAX; ++r) {
#pragma unroll
        for (int i = r & 1; i + 1 < KMAX; i += 2) {
            const float a = t[i], b = t[i + 1];
            t[i] = fminf(a, b);
            t[i + 1] = fmaxf(a, b);
        }
    }
}

// first index j in [lo, hi) with pred(j) true (pred monotone false -> true)
template <class Pred>
__device__ __forceinline__ int lower_search(int lo, int hi, Pred pred) {
    while (lo < hi) {
        const int mid = (lo + hi) >> 1;
        if (pred(mid)) hi = mid;
        else lo = mid + 1;
    }
    return lo;
}

__host__ __device__ constexpr size_t ksg_slot_bytes(int n_pad) {
    return (size_t)n_pad * (2 * sizeof(float2) + 2 * sizeof(uint16_t));
}

// Walk along sorted pairs W (walk value, other value) from position s.
// L / R = next unvisited positions on each side, dL / dR their axis distances
// (inf when exhausted), cL / cR their entries.
struct KsgWalk {
    const float2* W;
    int n, L, R;
    float pv, ov, dL, dR;
    float2 cL, cR;
    __device__ __forceinline__ void init(const float2* w, int n_, int s, float p, float o) {
        W = w;
        n = n_;
        pv = p;
        ov = o;
        L = s - 1;
        R = s + 1;
        cL = W[L >= 0 ? L : s];
        cR = W[R < n ? R : s];
        dL = L >= 0 ? __fsub_rn(pv, cL.x) : CUDART_INF_F;
        dR = R < n ? __fsub_rn(cR.x, pv) : CUDART_INF_F;
    }
    __device__ __forceinline__ float next_axis() const { return fminf(dL, dR); }
    // visit the nearer side's candidate (branch free); returns its Chebyshev distance
    __device__ __forceinline__ float step() {
        const bool right = dR < dL;
        const float da = right ? dR : dL;
        const float oj = right ? cR.y : cL.y;
        const float d = fmaxf(da, fabsf(__fsub_rn(ov, oj)));
        const int np = right ? R + 1 : L - 1;
        const bool inb = right ? np < n : np >= 0;
        const float2 c = W[inb ? np : (right ? R : L)];
        const float nd = !inb ? CUDART_INF_F : (right ? __fsub_rn(c.x, pv) : __fsub_rn(pv, c.x));
        if (right) {
            R = np;
            dR = nd;
            cR = c;
        } else {
            L = np;
            dL = nd;
            cL = c;
        }
        return d;
    }
};

// Warp-cooperative staging of one pair into a slot (ends with __syncwarp).
// sa/pa/va: sorted values, argsort and member values of point p (x);
// sb/pb/vb: the same for point q (y).
__device__ __forceinline__ void ksg_stage(unsigned char* slot, int n, int n_pad,
                                          const float* __restrict__ sa,
                                          const uint16_t* __restrict__ pa,
                                          const float* __restrict__ va,
                                          const float* __restrict__ sb,
                                          const uint16_t* __restrict__ pb,
                                          const float* __restrict__ vb) {
    const int lane = threadIdx.x & 31;
    float2* XO = reinterpret_cast<float2*>(slot);
    float2* YO = XO + n_pad;
    uint16_t* upos = reinterpret_cast<uint16_t*>(YO + n_pad);
    uint16_t* invq = upos + n_pad;
    for (int m = lane; m < n; m += 32) {
        const int mq = pb[m];
        invq[mq] = (uint16_t)m;
        YO[m] = make_float2(sb[m], va[mq]);
    }
    __syncwarp();
    for (int m = lane; m < n; m += 32) {
        const int mp = pa[m];
        XO[m] = make_float2(sa[m], vb[mp]);
        upos[m] = invq[mp];
    }
    __syncwarp();
}

// One sample (x-sorted position ti) of a staged pair: eps and the two counts;
// returns psi[n_x] + psi[n_y] from the fixed-point table.
template <int KMAX>
__device__ __forceinline__ long long ksg_sample(const unsigned char* slot, int n, int n_pad, int k,
                                                int ti, const long long* __restrict__ psi,
                                                int* cx_out, int* cy_out, float* eps_out) {
    const float2* XO = reinterpret_cast<const float2*>(slot);
    const float2* YO = XO + n_pad;
    const uint16_t* upos = reinterpret_cast<const uint16_t*>(YO + n_pad);
    const float2 zi = XO[ti];
    const int ui = upos[ti];
    // walk along the axis with the wider local spacing
    const int h = 4;
    const float span_x = __fsub_rn(XO[min(ti + h, n - 1)].x, XO[max(ti - h, 0)].x);
    const float span_y = __fsub_rn(YO[min(ui + h, n - 1)].x, YO[max(ui - h, 0)].x);
    const bool on_y = span_y > span_x;
    const float2* O = on_y ? XO : YO;  // other axis order (sorted in .x)
    const int s = on_y ? ui : ti;
    KsgWalk w;
    w.init(on_y ? YO : XO, n, s, on_y ? zi.y : zi.x, on_y ? zi.x : zi.y);
    float top[KMAX];
#pragma unroll
    for (int m = 0; m < KMAX; ++m)
        top[m] = m >= KMAX - k ? w.step() : -CUDART_INF_F;  // the k axis-nearest
    sort_net<KMAX>(top);
    while (w.next_axis() < top[KMAX - 1]) {
        const float d = w.step();
        if (d < top[KMAX - 1]) topk_insert<KMAX>(top, d);
    }
    const float eps = top[KMAX - 1];
    const float pv = w.pv, ov = w.ov;
    int L = w.L, R = w.R;
    // walk axis: trim the visited window (L, R) to axis distance < eps
    while (L + 1 < s && !(__fsub_rn(pv, w.W[L + 1].x) < eps)) ++L;
    while (R - 1 > s && !(__fsub_rn(w.W[R - 1].x, pv) < eps)) --R;
    const int c_walk = eps > 0.f ? R - L - 1 : 1;
    // other axis: [a, b) with a = first j with fl(ov - O[j].x) < eps,
    // b = first j with fl(O[j].x - ov) >= eps
    const int a = lower_search(0, n, [&](int j) { return __fsub_rn(ov, O[j].x) < eps; });
    const int b = lower_search(0, n, [&](int j) { return !(__fsub_rn(O[j].x, ov) < eps); });
    const int c_oth = max(b - a, 1);
    const int cx = on_y ? c_oth : c_walk;
    const int cy = on_y ? c_walk : c_oth;
    if (cx_out) {
        *cx_out = cx;
        *cy_out = cy;
        *eps_out = eps;
    }
    return psi[cx] + psi[cy];
}

}  // namespace cc
