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

// compare-exchange: a <- min, b <- max
__device__ __forceinline__ void ce(float& a, float& b) {
    const float lo = fminf(a, b);
    b = fmaxf(a, b);
    a = lo;
}

__host__ __device__ constexpr int ksg_pow2_at_least(int v) {
    int q = 1;
    while (q < v) q <<= 1;
    return q;
}

// ascending sort of a small register array. Fixed networks for the common
// sizes (4: 5 comparators; 8: 19; 10: 29, Waksman's network), a bitonic
// sorter for other powers of two, odd-even transposition otherwise. Each
// network is checked against all 0/1 inputs by a host test.
template <int N>
__device__ __forceinline__ void sort_small(float (&t)[N]) {
    if constexpr (N == 2) {
        ce(t[0], t[1]);
    } else if constexpr (N == 4) {
        ce(t[0], t[1]); ce(t[2], t[3]); ce(t[0], t[2]); ce(t[1], t[3]); ce(t[1], t[2]);
    } else if constexpr (N == 8) {
        ce(t[0], t[2]); ce(t[1], t[3]); ce(t[4], t[6]); ce(t[5], t[7]);
        ce(t[0], t[4]); ce(t[1], t[5]); ce(t[2], t[6]); ce(t[3], t[7]);
        ce(t[0], t[1]); ce(t[2], t[3]); ce(t[4], t[5]); ce(t[6], t[7]);
        ce(t[2], t[4]); ce(t[3], t[5]); ce(t[1], t[4]); ce(t[3], t[6]);
        ce(t[1], t[2]); ce(t[3], t[4]); ce(t[5], t[6]);
    } else if constexpr (N == 10) {
        ce(t[4], t[9]); ce(t[3], t[8]); ce(t[2], t[7]); ce(t[1], t[6]); ce(t[0], t[5]);
        ce(t[1], t[4]); ce(t[6], t[9]); ce(t[0], t[3]); ce(t[5], t[8]); ce(t[0], t[2]);
        ce(t[3], t[6]); ce(t[7], t[9]); ce(t[0], t[1]); ce(t[2], t[4]); ce(t[5], t[7]);
        ce(t[8], t[9]); ce(t[1], t[2]); ce(t[4], t[6]); ce(t[7], t[8]); ce(t[3], t[5]);
        ce(t[2], t[5]); ce(t[6], t[8]); ce(t[1], t[3]); ce(t[4], t[7]); ce(t[2], t[3]);
        ce(t[6], t[7]); ce(t[3], t[4]); ce(t[5], t[6]); ce(t[4], t[5]);
    } else if constexpr (ksg_pow2_at_least(N) == N) {
#pragma unroll
        for (int size = 2; size <= N; size *= 2) {
#pragma unroll
            for (int stride = size / 2; stride > 0; stride /= 2) {
#pragma unroll
                for (int i = 0; i < N; ++i) {
                    const int j = i ^ stride;
                    if (j > i) {
                        if ((i & size) == 0) ce(t[i], t[j]);
                        else ce(t[j], t[i]);
                    }
                }
            }
        }
    } else {
#pragma unroll
        for (int r = 0; r < N; ++r) {
#pragma unroll
            for (int i = r & 1; i + 1 < N; i += 2) ce(t[i], t[i + 1]);
        }
    }
}

// Sort a bitonic register array (ascending then descending) ascending: the
// bitonic merger of the next power of two Q, with Q - KMAX virtual -inf
// entries in front (comparators touching them are no-ops and are dropped).
template <int KMAX>
__device__ __forceinline__ void bitonic_merge(float (&t)[KMAX]) {
    constexpr int Q = ksg_pow2_at_least(KMAX), PADN = Q - KMAX;
#pragma unroll
    for (int d = Q / 2; d > 0; d /= 2) {
#pragma unroll
        for (int q = PADN; q < Q; ++q)
            if ((q & d) == 0) ce(t[q - PADN], t[q + d - PADN]);
    }
}

// The KMAX smallest of the sorted list t and four new values, sorted: the
// new values are sorted, the i-th largest list entry is replaced by the
// minimum of itself and the i-th smallest new value (the result holds the
// KMAX smallest and is bitonic), and a bitonic merger restores the order.
template <int KMAX>
__device__ __forceinline__ void topk_merge4(float (&t)[KMAX], float c0, float c1, float c2,
                                            float c3) {
    if constexpr (KMAX < 4) {
        topk_insert<KMAX>(t, c0);
        topk_insert<KMAX>(t, c1);
        topk_insert<KMAX>(t, c2);
        topk_insert<KMAX>(t, c3);
    } else {
        float c[4] = {c0, c1, c2, c3};
        sort_small<4>(c);
#pragma unroll
        for (int j = 0; j < 4; ++j) t[KMAX - 1 - j] = fminf(t[KMAX - 1 - j], c[j]);
        bitonic_merge<KMAX>(t);
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

// KMAX instantiated for a given k (the list length rounded up to a template size)
__host__ __device__ constexpr int ksg_kmax(int k) {
    return k <= 1 ? 1 : k == 2 ? 2 : k == 3 ? 3 : k <= 4 ? 4 : k <= 8 ? 8 : k <= 10 ? 10
           : k <= 16 ? 16 : 32;
}

// sentinel entries on each side of a staged sorted array: the walk's start
// reads up to ceil(KMAX/2) positions out, a step up to seven positions past
// the next position of an open side, and the window trim up to seven
// positions past the sample
__host__ __device__ constexpr int ksg_pad(int kmax) {
    return (kmax + 1) / 2 + 2 > 7 ? (kmax + 1) / 2 + 2 : 7;
}

__host__ __device__ constexpr size_t ksg_slot_bytes(int n_pad, int kmax) {
    return (size_t)(n_pad + 2 * ksg_pad(kmax)) * 2 * sizeof(float2) +
           (size_t)n_pad * 2 * sizeof(uint16_t);
}

// Warp-cooperative staging of one pair into a slot (ends with __syncwarp).
// sa/pa/va: sorted values, argsort and member values of point p (x);
// sb/pb/vb: the same for point q (y). Both sorted arrays get ksg_pad(KMAX)
// sentinels per side, -inf on the left and +inf on the right, so that every
// axis distance to a sentinel is +inf. Members are taken 128 at a time (four
// per lane): every global load of a batch is issued before the gathers that
// depend on it, so a batch costs two memory round trips.
template <int KMAX>
__device__ __forceinline__ void ksg_stage(unsigned char* slot, int n, int n_pad,
                                          const float* __restrict__ sa,
                                          const uint16_t* __restrict__ pa,
                                          const float* __restrict__ va,
                                          const float* __restrict__ sb,
                                          const uint16_t* __restrict__ pb,
                                          const float* __restrict__ vb) {
    constexpr int pad = ksg_pad(KMAX);
    constexpr int IT = 4;
    const int lane = threadIdx.x & 31;
    float2* XO = reinterpret_cast<float2*>(slot) + pad;
    float2* YO = XO + n_pad + 2 * pad;
    uint16_t* upos = reinterpret_cast<uint16_t*>(YO + n_pad + pad);
    uint16_t* invq = upos + n_pad;
    // -inf before position 0; +inf from position n up to n_pad + pad - 1
    // (the counting search of ksg_finish probes up to position n_pad - 1)
    const float2 lo = make_float2(-CUDART_INF_F, 0.f), hi = make_float2(CUDART_INF_F, 0.f);
    if (lane < pad) {
        XO[lane - pad] = lo;
        YO[lane - pad] = lo;
    }
    for (int j = n + lane; j < n_pad + pad; j += 32) {
        XO[j] = hi;
        YO[j] = hi;
    }
    // y side: invq (inverse argsort of q) and YO = (y sorted, x of that member)
    for (int base = 0; base < n; base += 32 * IT) {
        int mq[IT];
        float y[IT], x[IT];
#pragma unroll
        for (int i = 0; i < IT; ++i) {
            const int m = base + 32 * i + lane;
            mq[i] = m < n ? pb[m] : 0;
            y[i] = m < n ? sb[m] : 0.f;
        }
#pragma unroll
        for (int i = 0; i < IT; ++i) x[i] = base + 32 * i + lane < n ? va[mq[i]] : 0.f;
#pragma unroll
        for (int i = 0; i < IT; ++i) {
            const int m = base + 32 * i + lane;
            if (m < n) {
                invq[mq[i]] = (uint16_t)m;
                YO[m] = make_float2(y[i], x[i]);
            }
        }
    }
    __syncwarp();
    // x side: XO = (x sorted, y of that member), upos = y-sorted position
    for (int base = 0; base < n; base += 32 * IT) {
        int mp[IT];
        float x[IT], y[IT];
#pragma unroll
        for (int i = 0; i < IT; ++i) {
            const int m = base + 32 * i + lane;
            mp[i] = m < n ? pa[m] : 0;
            x[i] = m < n ? sa[m] : 0.f;
        }
#pragma unroll
        for (int i = 0; i < IT; ++i) y[i] = base + 32 * i + lane < n ? vb[mp[i]] : 0.f;
#pragma unroll
        for (int i = 0; i < IT; ++i) {
            const int m = base + 32 * i + lane;
            if (m < n) {
                XO[m] = make_float2(x[i], y[i]);
                upos[m] = invq[mp[i]];
            }
        }
    }
    __syncwarp();
}

// The walk state of one sample of a staged pair (ksg_begin, ksg_step,
// ksg_finish below; ksg_sample runs them in order).
//
// The walk runs along one axis (W: that axis's sorted (value, other value)
// entries), from the sample's position s outwards on both sides at once.
// L / R are the next unvisited positions on each side. The first k
// positions (ceil(k/2) left, floor(k/2) right) are visited unconditionally
// and sorted; the first step offers the next four positions of each side
// (ksg_step8), every later step the next two (ksg_step), and a step advances
// a side past the positions whose axis distance was below the k-th smallest
// value before the step. A position that is offered but not
// passed has a Chebyshev distance not below that value, so it cannot change
// the list (and it is offered again only under the same condition). The
// walk ends when both next axis distances are not below the k-th smallest
// value; every position not passed then has a distance not below it, so the
// list's last entry is eps exactly.
template <int KMAX>
struct KsgWalk {
    float top[KMAX];    // the KMAX smallest distances offered so far, ascending
    const float2* W;    // walk axis order
    const float2* O;    // other axis order (sorted in .x)
    float pv, ov;       // the sample's value on the walk / other axis
    int s, L, R;        // the sample's walk position; next unvisited positions
    bool on_y;          // the walk runs along y
};

// Start the walk of sample ti (x-sorted position) of a staged pair: choose
// the axis, visit the first k positions and sort them.
template <int KMAX>
__device__ __forceinline__ void ksg_begin(KsgWalk<KMAX>& w, const unsigned char* slot, int n,
                                          int n_pad, int k, int ti) {
    constexpr int pad = ksg_pad(KMAX);
    constexpr int P1 = (KMAX + 1) / 2, NP1 = 2 * P1;
    const float2* XO = reinterpret_cast<const float2*>(slot) + pad;
    const float2* YO = XO + n_pad + 2 * pad;
    const uint16_t* upos = reinterpret_cast<const uint16_t*>(YO + n_pad + pad);
    const float2 zi = XO[ti];
    const int ui = upos[ti];
    // Walk along the axis on which fewer samples lie within eps. The walk
    // visits about as many positions as its axis has samples closer than
    // eps, typically sqrt(k n) of them, so each axis is scored by the radius
    // around the sample that holds m ~ 0.8 sqrt(k n) sorted positions: for
    // two placements of a window of m + 1 consecutive positions that
    // contains the sample (clipped to the sorted order), the larger of the
    // window's two end distances; the smaller over the placements estimates
    // the radius of the m nearest positions, and the axis with the larger
    // radius is walked. (A wrong choice costs steps, never exactness.)
    const int m = min((int)(0.8f * sqrtf((float)(k * n)) + 0.5f), n - 1);
    auto window = [&](const float2* A, int r, float v, int j) {
        const int lo = min(max(r - j, 0), n - 1 - m);
        return fmaxf(__fsub_rn(v, A[lo].x), __fsub_rn(A[lo + m].x, v));
    };
    const float rad_x = fminf(window(XO, ti, zi.x, m >> 2), window(XO, ti, zi.x, (3 * m) >> 2));
    const float rad_y = fminf(window(YO, ui, zi.y, m >> 2), window(YO, ui, zi.y, (3 * m) >> 2));
    w.on_y = rad_y > rad_x;
    w.W = w.on_y ? YO : XO;
    w.O = w.on_y ? XO : YO;
    w.s = w.on_y ? ui : ti;
    w.pv = w.on_y ? zi.y : zi.x;
    w.ov = w.on_y ? zi.x : zi.y;
    // the first k positions, alternating left / right; unused slots are -inf
    float c[NP1];
#pragma unroll
    for (int t = 0; t < P1; ++t) {
        const float2 l = w.W[w.s - 1 - t], r = w.W[w.s + 1 + t];
        const float dl = fmaxf(__fsub_rn(w.pv, l.x), fabsf(__fsub_rn(w.ov, l.y)));
        const float dr = fmaxf(__fsub_rn(r.x, w.pv), fabsf(__fsub_rn(w.ov, r.y)));
        c[2 * t] = dl;
        c[2 * t + 1] = dr;
    }
    if (k < NP1) {  // the same for every lane
#pragma unroll
        for (int t = 0; t < NP1; ++t)
            if (t >= k) c[t] = -CUDART_INF_F;
    }
    sort_small<NP1>(c);
#pragma unroll
    for (int m = 0; m < KMAX; ++m) w.top[m] = c[m + NP1 - KMAX];
    w.L = w.s - (k + 1) / 2 - 1;
    w.R = w.s + k / 2 + 1;
}

// One walk step; returns false (and changes nothing) once the walk has ended.
template <int KMAX>
__device__ __forceinline__ bool ksg_step(KsgWalk<KMAX>& w) {
    // a side is open while its next axis distance is below the k-th value;
    // a step offers two positions per open side, or four from the only open
    // side (a walk near either end of the sorted order then takes half the
    // steps). Offered positions: L, L-1 (or R+2, R+3 when the left side is
    // closed) and R, R+1 (or L-2, L-3 when the right side is closed); an
    // open left side has L >= 0 and an open right side R <= n - 1, so every
    // index stays within the sentinels.
    const float2* W = w.W;
    const int L = w.L, R = w.R;
    const float pv = w.pv, ov = w.ov;
    const float kth = w.top[KMAX - 1];
    const float2 wl = W[L], wr = W[R];
    const bool lo = __fsub_rn(pv, wl.x) < kth;
    const bool ro = __fsub_rn(wr.x, pv) < kth;
    if (!(lo || ro)) return false;
    const float2 z0 = lo ? wl : W[R + 2], z1 = W[lo ? L - 1 : R + 3];
    const float2 z2 = ro ? wr : W[L - 2], z3 = W[ro ? R + 1 : L - 3];
    const float a0 = fabsf(__fsub_rn(pv, z0.x)), a1 = fabsf(__fsub_rn(pv, z1.x));
    const float a2 = fabsf(__fsub_rn(pv, z2.x)), a3 = fabsf(__fsub_rn(pv, z3.x));
    const float d0 = fmaxf(a0, fabsf(__fsub_rn(ov, z0.y)));
    const float d1 = fmaxf(a1, fabsf(__fsub_rn(ov, z1.y)));
    const float d2 = fmaxf(a2, fabsf(__fsub_rn(ov, z2.y)));
    const float d3 = fmaxf(a3, fabsf(__fsub_rn(ov, z3.y)));
    // positions are passed in order of axis distance on each side, so the
    // passed ones of z0, z1 and of z2, z3 are prefixes
    const int c01 = (int)(a0 < kth) + (int)(a1 < kth);
    const int c23 = (int)(a2 < kth) + (int)(a3 < kth);
    w.L = L - (lo ? c01 + (ro ? 0 : c23) : 0);
    w.R = R + (ro ? c23 + (lo ? 0 : c01) : 0);
    topk_merge4<KMAX>(w.top, d0, d1, d2, d3);
    return true;
}

// The KMAX smallest of the sorted list t and eight new values, sorted (as
// topk_merge4, with a sorting network of eight).
template <int KMAX>
__device__ __forceinline__ void topk_merge8(float (&t)[KMAX], float (&c)[8]) {
    sort_small<8>(c);
    if constexpr (KMAX >= 8) {
#pragma unroll
        for (int j = 0; j < 8; ++j) t[KMAX - 1 - j] = fminf(t[KMAX - 1 - j], c[j]);
        bitonic_merge<KMAX>(t);
    } else {
#pragma unroll
        for (int j = 0; j < 8; ++j) topk_insert<KMAX>(t, c[j]);
    }
}

// The first step after ksg_begin: as ksg_step, with four positions per open
// side, or eight from the only open side. Almost every walk takes at least
// two steps, so this merges the first two into one with one sorting network
// of eight. An open left side has L >= 0 and an open right side R <= n - 1,
// so every index stays within seven positions of the sorted order, inside
// the sentinels.
template <int KMAX>
__device__ __forceinline__ bool ksg_step8(KsgWalk<KMAX>& w) {
    const float2* W = w.W;
    const int L = w.L, R = w.R;
    const float pv = w.pv, ov = w.ov;
    const float kth = w.top[KMAX - 1];
    const float2 wl = W[L], wr = W[R];
    const bool lo = __fsub_rn(pv, wl.x) < kth;
    const bool ro = __fsub_rn(wr.x, pv) < kth;
    if (!(lo || ro)) return false;
    float c[8];
    int cl = 0, cr = 0;
#pragma unroll
    for (int j = 0; j < 4; ++j) {
        // left offers L - j (or R + 4 + j when closed), right R + j (or L - 4 - j)
        const float2 zl = j == 0 && lo ? wl : W[lo ? L - j : R + 4 + j];
        const float2 zr = j == 0 && ro ? wr : W[ro ? R + j : L - 4 - j];
        const float al = fabsf(__fsub_rn(pv, zl.x)), ar = fabsf(__fsub_rn(pv, zr.x));
        c[j] = fmaxf(al, fabsf(__fsub_rn(ov, zl.y)));
        c[4 + j] = fmaxf(ar, fabsf(__fsub_rn(ov, zr.y)));
        cl += (int)(al < kth);
        cr += (int)(ar < kth);
    }
    // passed positions are prefixes of each side (axis distance grows outwards)
    w.L = L - (lo ? cl + (ro ? 0 : cr) : 0);
    w.R = R + (ro ? cr + (lo ? 0 : cl) : 0);
    topk_merge8<KMAX>(w.top, c);
    return true;
}

// One level of the counting search of ksg_finish: the probes at offset
// H - 1 from the lower bound a and the upper bound b.
template <int H>
__device__ __forceinline__ void ksg_probe2(const float2* O, int& a, int& b, float ov, float eps) {
    if (!(__fsub_rn(ov, O[a + (H - 1)].x) < eps)) a += H;
    if (__fsub_rn(O[b + (H - 1)].x, ov) < eps) b += H;
}

// The counts of a finished walk; returns psi[n_x] + psi[n_y] from the
// fixed-point table.
template <int KMAX>
__device__ __forceinline__ long long ksg_finish(const KsgWalk<KMAX>& w, int n,
                                                const long long* __restrict__ psi, int* cx_out,
                                                int* cy_out, float* eps_out) {
    const float2* W = w.W;
    const float2* O = w.O;
    const float pv = w.pv, ov = w.ov, eps = w.top[KMAX - 1];
    const int s = w.s;
    // walk axis: the passed window (L, R), trimmed to axis distance < eps.
    // Along each side the axis distance falls towards s, so the positions to
    // trim are a prefix of the side; almost always fewer than eight, found
    // by lifting over 4, 2, 1, with a position-by-position continuation
    // beyond seven. The lifting needs no window bound: for eps > 0 the
    // sample's own position and everything past it (sentinels included)
    // fail the trim test, and the probes stay within seven positions of the
    // window, inside the sentinels (for eps = 0 the count is 1 whatever the
    // trim finds).
    int L = max(w.L, -1), R = min(w.R, n);
    {
        const int wl = s - 1 - L, wr = R - 1 - s;
        int tl = 0, tr = 0;
#pragma unroll
        for (int step = 4; step > 0; step >>= 1) {
            if (!(__fsub_rn(pv, W[L + tl + step].x) < eps)) tl += step;
            if (!(__fsub_rn(W[R - tr - step].x, pv) < eps)) tr += step;
        }
        if (tl == 7)
            while (tl < wl && !(__fsub_rn(pv, W[L + tl + 1].x) < eps)) ++tl;
        if (tr == 7)
            while (tr < wr && !(__fsub_rn(W[R - tr - 1].x, pv) < eps)) ++tr;
        L += tl;
        R -= tr;
    }
    const int c_walk = eps > 0.f ? R - L - 1 : 1;
    // other axis: [a, b) with a = first j with fl(ov - O[j].x) < eps,
    // b = first j with fl(O[j].x - ov) >= eps (fl32 differences are monotone
    // along the sorted order; the +inf entries from position n on satisfy
    // both tests, so a, b <= n). Both by one branch-free search (a and b
    // interleaved) over a range of 2^L >= n positions: the answer lies in
    // [base, base + len], a probe at base + len / 2 - 1 either moves base up
    // by len / 2 or leaves it, and len halves. L is the same for every lane,
    // so the probes are unrolled with constant offsets from the entry point
    // that L selects, and no probe passes position 2^L - 1 <= n_pad - 1.
    int a = 0, b = 0;
    switch (32 - __clz(n - 1)) {  // L = ceil(log2 n), 1 <= L <= 10 for 2 <= n <= 1024
        case 10: ksg_probe2<512>(O, a, b, ov, eps); [[fallthrough]];
        case 9: ksg_probe2<256>(O, a, b, ov, eps); [[fallthrough]];
        case 8: ksg_probe2<128>(O, a, b, ov, eps); [[fallthrough]];
        case 7: ksg_probe2<64>(O, a, b, ov, eps); [[fallthrough]];
        case 6: ksg_probe2<32>(O, a, b, ov, eps); [[fallthrough]];
        case 5: ksg_probe2<16>(O, a, b, ov, eps); [[fallthrough]];
        case 4: ksg_probe2<8>(O, a, b, ov, eps); [[fallthrough]];
        case 3: ksg_probe2<4>(O, a, b, ov, eps); [[fallthrough]];
        case 2: ksg_probe2<2>(O, a, b, ov, eps); [[fallthrough]];
        default: ksg_probe2<1>(O, a, b, ov, eps);
    }
    a += !(__fsub_rn(ov, O[a].x) < eps) ? 1 : 0;
    b += __fsub_rn(O[b].x, ov) < eps ? 1 : 0;
    const int c_oth = max(b - a, 1);
    const int cx = w.on_y ? c_oth : c_walk;
    const int cy = w.on_y ? c_walk : c_oth;
    if (cx_out) {
        *cx_out = cx;
        *cy_out = cy;
        *eps_out = eps;
    }
    return psi[cx] + psi[cy];
}

// One sample (x-sorted position ti) of a staged pair: eps and the two counts;
// returns psi[n_x] + psi[n_y] from the fixed-point table. kLong: every step
// offers eight positions (long walks, n > 256); otherwise only the first.
template <int KMAX, bool kLong = false>
__device__ __forceinline__ long long ksg_sample(const unsigned char* slot, int n, int n_pad, int k,
                                                int ti, const long long* __restrict__ psi,
                                                int* cx_out, int* cy_out, float* eps_out) {
    KsgWalk<KMAX> w;
    ksg_begin<KMAX>(w, slot, n, n_pad, k, ti);
    if constexpr (kLong) {
        while (ksg_step8<KMAX>(w)) {
        }
    } else if (ksg_step8<KMAX>(w)) {
        while (ksg_step<KMAX>(w)) {
        }
    }
    return ksg_finish<KMAX>(w, n, psi, cx_out, cy_out, eps_out);
}

}  // namespace cc
