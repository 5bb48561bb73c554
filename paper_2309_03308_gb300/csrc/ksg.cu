// Kraskov (KSG) mutual information on a batch of point pairs (Section 3.2).
//
// For a pair (p, q) the joint samples are z_i = (x_i, y_i), x = members of
// p, y = members of q. With fp32 differences (bit-identical to the
// definition):
//   eps_i = k-th smallest d_ij = max(|x_i - x_j|, |y_i - y_j|) over j != i
//   n_x,i = 1 + #{j != i : |x_i - x_j| < eps_i}, n_y,i likewise
//   MI    = psi(n) + psi(k) - (1/n) sum_i [psi(n_x,i) + psi(n_y,i)]
//
// Design (one warp per group of up to 4 pairs, one lane per sample i):
//   For each pair the warp stages (x, y) in x-sorted order, (y, x) in
//   y-sorted order and each sample's y-sorted position in shared memory; the
//   per-point sorted values and argsorts come from ingest, so staging is
//   gathers only. The samples of the group's pairs form one stream that the
//   lanes take 32 at a time, so no lane idles at the end of a pair.
//
//   eps_i: walk outward from i along ONE axis in non-decreasing axis distance
//   (two pointers over that axis's sorted order); every visited j offers d_ij.
//   The first k visited are taken unconditionally and sorted once; later ones
//   enter a sorted register list of the k smallest. When the next axis
//   distance is not below the current k-th value no later j can enter, so the
//   walk stops with the exact k-th smallest. The walk length is about the
//   number of samples within eps_i along the axis, large where that axis is
//   locally dense; each lane walks along the axis whose local spacing
//   (8-neighbour span in sorted order) is wider. The step is branch-free and
//   all lanes run the same code on lane-selected arrays.
//
//   Counts: the walk's final window holds every j with axis distance below
//   eps_i (trimmed at its ends); the other axis is counted with two binary
//   searches on its sorted values (fl32 differences are monotone, so the set
//   is a contiguous range). The self sample is in the range exactly when
//   eps_i > 0, giving 1 + #{j != i} as defined.
//
//   The digamma sum uses a fixed-point table (2^-40), exact and order
//   independent; psi(n) + psi(k) and the final scaling are FP64.
#include "device.cuh"
#include "internal.cuh"

namespace cc {

double digamma_int_host(int m);

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

constexpr int kKsgWarps = 4;
constexpr int kMaxGroup = 4;

__host__ __device__ constexpr size_t ksg_slot_bytes(int n_pad) {
    return (size_t)n_pad * (2 * sizeof(float2) + 2 * sizeof(uint16_t));
}

// One walk along sorted pairs W (walk value, other value) from position s.
// State: L / R = next unvisited positions on each side, dL / dR their axis
// distances (inf when exhausted), cL / cR their entries.
struct Walk {
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
    // visit the nearer side's candidate; returns its Chebyshev distance
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

template <int KMAX>
__global__ void __launch_bounds__(kKsgWarps * 32)
    k_ksg_pairs(const float* __restrict__ sorted_a, const uint16_t* __restrict__ perm_a,
                const float* __restrict__ vals_a, int64_t Pa, const float* __restrict__ sorted_b,
                const uint16_t* __restrict__ perm_b, const float* __restrict__ vals_b, int64_t Pb,
                int n, int n_pad, int k, int G, const long long* __restrict__ psi_fix,
                double psi_nk, const uint32_t* __restrict__ pa, const uint32_t* __restrict__ pb,
                int64_t N, float* __restrict__ out, int32_t* __restrict__ nx_out,
                int32_t* __restrict__ ny_out, float* __restrict__ eps_out, int* status) {
    extern __shared__ __align__(16) unsigned char ksg_smem[];
    long long* psi = reinterpret_cast<long long*>(ksg_smem);
    const int psi_len = (n + 2) & ~1;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const size_t slot_bytes = ksg_slot_bytes(n_pad);
    unsigned char* wbase = ksg_smem + psi_len * sizeof(long long) + (size_t)warp * G * slot_bytes;
    for (int i = threadIdx.x; i <= n; i += blockDim.x) psi[i] = psi_fix[i];
    __syncthreads();

    const int64_t ngroups = (N + G - 1) / G;
    for (int64_t g = (int64_t)blockIdx.x * kKsgWarps + warp; g < ngroups;
         g += (int64_t)gridDim.x * kKsgWarps) {
        const int64_t t0 = g * G;
        const int gc = (int)min((int64_t)G, N - t0);
        unsigned valid = 0;
        for (int sl = 0; sl < gc; ++sl) {
            const uint32_t p = pa[t0 + sl], q = pb[t0 + sl];
            if (p >= Pa || q >= Pb) {
                if (lane == 0) {
                    out[t0 + sl] = CUDART_NAN_F;
                    set_status(status, DEV_BAD_INDEX);
                }
                continue;
            }
            valid |= 1u << sl;
            unsigned char* b = wbase + sl * slot_bytes;
            float2* XO = reinterpret_cast<float2*>(b);
            float2* YO = XO + n_pad;
            uint16_t* upos = reinterpret_cast<uint16_t*>(YO + n_pad);
            uint16_t* invq = upos + n_pad;
            const int64_t ra = (int64_t)p * n_pad, rb = (int64_t)q * n_pad;
            for (int m = lane; m < n; m += 32) {
                const int mq = perm_b[rb + m];
                invq[mq] = (uint16_t)m;
                YO[m] = make_float2(sorted_b[rb + m], vals_a[ra + mq]);
            }
            __syncwarp();
            for (int m = lane; m < n; m += 32) {
                const int mp = perm_a[ra + m];
                XO[m] = make_float2(sorted_a[ra + m], vals_b[rb + mp]);
                upos[m] = invq[mp];
            }
        }
        __syncwarp();

        long long acc[kMaxGroup];
#pragma unroll
        for (int u = 0; u < kMaxGroup; ++u) acc[u] = 0;
        const int items = gc * n;
        for (int it = lane; it < items; it += 32) {
            const int sl = it / n, ti = it - sl * n;
            if (!((valid >> sl) & 1u)) continue;
            unsigned char* b = wbase + sl * slot_bytes;
            const float2* XO = reinterpret_cast<const float2*>(b);
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
            Walk w;
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
            const int bb =
                lower_search(0, n, [&](int j) { return !(__fsub_rn(O[j].x, ov) < eps); });
            const int c_oth = max(bb - a, 1);
            const int cx = on_y ? c_oth : c_walk;
            const int cy = on_y ? c_walk : c_oth;
            const long long v = psi[cx] + psi[cy];
#pragma unroll
            for (int u = 0; u < kMaxGroup; ++u)
                if (u == sl) acc[u] += v;
            if (nx_out) {
                const int64_t t = t0 + sl;
                const int orig = perm_a[(int64_t)pa[t] * n_pad + ti];
                nx_out[t * n + orig] = cx;
                ny_out[t * n + orig] = cy;
                if (eps_out) eps_out[t * n + orig] = eps;
            }
        }
#pragma unroll
        for (int u = 0; u < kMaxGroup; ++u) {
            if (u < gc) {
                const long long sum = warp_sum_i64(acc[u]);
                if (lane == 0 && ((valid >> u) & 1u))
                    out[t0 + u] = (float)(psi_nk - ((double)sum / kFixScale) / (double)n);
            }
        }
        __syncwarp();
    }
}

template <int KMAX>
static cudaError_t ksg_launch(const Field& fa, const Field& fb, int k, const int64_t* psi_fix,
                              double psi_nk, const uint32_t* pa, const uint32_t* pb, int64_t N,
                              float* out, int32_t* nx, int32_t* ny, float* eps, int* status,
                              cudaStream_t st) {
    // two pairs per warp while n is small, so the sample stream fills the lanes
    // (more pairs per warp costs occupancy through shared memory)
    const int G = fa.n_pad <= 128 ? 2 : 1;
    const int psi_len = (fa.n + 2) & ~1;
    const size_t smem = psi_len * sizeof(long long) + kKsgWarps * G * ksg_slot_bytes(fa.n_pad);
    if (smem > 48 * 1024) {
        cudaError_t e = cudaFuncSetAttribute(k_ksg_pairs<KMAX>,
                                             cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             (int)smem);
        if (e != cudaSuccess) return e;
    }
    int dev = 0, sms = 148;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    const int64_t groups = (N + G - 1) / G;
    int64_t blocks = (groups + kKsgWarps - 1) / kKsgWarps;
    blocks = blocks < (int64_t)sms * 16 ? blocks : (int64_t)sms * 16;
    note_launch();
    k_ksg_pairs<KMAX><<<(unsigned)blocks, kKsgWarps * 32, smem, st>>>(
        fa.sorted.as<float>(), fa.perm.as<uint16_t>(), fa.vals.as<float>(), fa.P,
        fb.sorted.as<float>(), fb.perm.as<uint16_t>(), fb.vals.as<float>(), fb.P, fa.n, fa.n_pad,
        k, G, (const long long*)psi_fix, psi_nk, pa, pb, N, out, nx, ny, eps, status);
    return cudaGetLastError();
}

cudaError_t launch_ksg_pairs(const Field& fa, const Field& fb, int k, const int64_t* psi_fix,
                             const uint32_t* pa, const uint32_t* pb, int64_t N, float* out,
                             int32_t* nx, int32_t* ny, float* eps, int* status, cudaStream_t st) {
    if (N <= 0) return cudaSuccess;
    const double psi_nk = digamma_int_host(fa.n) + digamma_int_host(k);
#define CC_KSG(KM) \
    return ksg_launch<KM>(fa, fb, k, psi_fix, psi_nk, pa, pb, N, out, nx, ny, eps, status, st)
    if (k <= 1) CC_KSG(1);
    if (k == 2) CC_KSG(2);
    if (k == 3) CC_KSG(3);
    if (k == 4) CC_KSG(4);
    if (k <= 8) CC_KSG(8);
    if (k <= 10) CC_KSG(10);
    if (k <= 16) CC_KSG(16);
    CC_KSG(32);
#undef CC_KSG
}

}  // namespace cc
