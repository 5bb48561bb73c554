// Kraskov (KSG) mutual information on a batch of point pairs (Section 3.2).
//
// For a pair (p, q) the joint samples are z_i = (x_i, y_i), x = members of
// p, y = members of q. With fp32 differences (bit-identical to the
// definition):
//   eps_i = k-th smallest d_ij = max(|x_i - x_j|, |y_i - y_j|) over j != i
//   n_x,i = 1 + #{j != i : |x_i - x_j| < eps_i}, n_y,i likewise
//   MI    = psi(n) + psi(k) - (1/n) sum_i [psi(n_x,i) + psi(n_y,i)]
//
// Design (one warp per pair, one lane per sample i):
//   The warp stages four views of the pair in shared memory: xs (x sorted),
//   ys (y in x-sorted order), sy (y sorted), xsy (x in y-sorted order), plus
//   each sample's position in y-sorted order. Per-point sorted values and
//   argsorts come precomputed from ingest, so staging is gathers only.
//
//   eps_i: walk outward from i along ONE axis in non-decreasing |d_axis|
//   (two pointers over that axis's sorted order); every visited j offers
//   d_ij to a sorted register list of the K smallest. When the next axis
//   distance is not below the current K-th value no later j can enter, so
//   the walk stops with the exact k-th smallest. The walk length is about
//   the number of samples within eps_i along the axis, which is large where
//   that axis is locally dense; each lane therefore walks along the axis
//   whose local spacing (8-neighbour span in sorted order) is wider. All
//   lanes run the same loop on lane-selected arrays, so the choice itself
//   costs no divergence.
//
//   Counts: the walk's final window contains every j with axis distance
//   below eps_i (trimmed at its ends); the other axis is counted with two
//   binary searches on its sorted values (fl32 differences are monotone, so
//   the qualifying set is a contiguous range). The self sample is in the
//   range exactly when eps_i > 0, giving 1 + #{j != i} as defined.
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

__host__ __device__ constexpr size_t ksg_warp_bytes(int n_pad) {
    return (size_t)n_pad * (4 * sizeof(float) + 2 * sizeof(uint16_t));
}

template <int KMAX>
__global__ void __launch_bounds__(kKsgWarps * 32)
    k_ksg_pairs(const float* __restrict__ sorted_a, const uint16_t* __restrict__ perm_a,
                const float* __restrict__ vals_a, int64_t Pa, const float* __restrict__ sorted_b,
                const uint16_t* __restrict__ perm_b, const float* __restrict__ vals_b, int64_t Pb,
                int n, int n_pad, int k, const long long* __restrict__ psi_fix, double psi_nk,
                const uint32_t* __restrict__ pa, const uint32_t* __restrict__ pb, int64_t N,
                float* __restrict__ out, int32_t* __restrict__ nx_out,
                int32_t* __restrict__ ny_out, float* __restrict__ eps_out, int* status) {
    extern __shared__ __align__(16) unsigned char ksg_smem[];
    long long* psi = reinterpret_cast<long long*>(ksg_smem);
    const int psi_len = (n + 2) & ~1;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    unsigned char* wbase =
        ksg_smem + psi_len * sizeof(long long) + (size_t)warp * ksg_warp_bytes(n_pad);
    // XO[t] = (x, y) of the sample at x-sorted position t (x ascending);
    // YO[u] = (y, x) of the sample at y-sorted position u (y ascending).
    float2* XO = reinterpret_cast<float2*>(wbase);
    float2* YO = XO + n_pad;
    uint16_t* upos = reinterpret_cast<uint16_t*>(YO + n_pad);
    uint16_t* invq = upos + n_pad;
    for (int i = threadIdx.x; i <= n; i += blockDim.x) psi[i] = psi_fix[i];
    __syncthreads();

    const int64_t w0 = (int64_t)blockIdx.x * kKsgWarps + warp;
    const int64_t stride = (int64_t)gridDim.x * kKsgWarps;
    for (int64_t t = w0; t < N; t += stride) {
        const uint32_t p = pa[t], q = pb[t];
        if (p >= Pa || q >= Pb) {
            if (lane == 0) {
                out[t] = CUDART_NAN_F;
                set_status(status, DEV_BAD_INDEX);
            }
            continue;
        }
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
        __syncwarp();

        long long acc = 0;
        for (int ti = lane; ti < n; ti += 32) {
            const float2 zi = XO[ti];
            const int ui = upos[ti];
            // axis choice: walk along the axis with the wider local spacing
            const int h = 4;
            const float span_x = __fsub_rn(XO[min(ti + h, n - 1)].x, XO[max(ti - h, 0)].x);
            const float span_y = __fsub_rn(YO[min(ui + h, n - 1)].x, YO[max(ui - h, 0)].x);
            const bool on_y = span_y > span_x;
            const float2* W = on_y ? YO : XO;  // walk order: (walk value, other value)
            const float2* O = on_y ? XO : YO;  // other axis order (sorted in .x)
            const int s = on_y ? ui : ti;
            const float pv = on_y ? zi.y : zi.x, ov = on_y ? zi.x : zi.y;

            float top[KMAX];
#pragma unroll
            for (int m = 0; m < KMAX; ++m) top[m] = m < KMAX - k ? -CUDART_INF_F : CUDART_INF_F;
            int L = s - 1, R = s + 1;
            float2 cL = L >= 0 ? W[L] : make_float2(0.f, 0.f);
            float2 cR = R < n ? W[R] : make_float2(0.f, 0.f);
            float dL = L >= 0 ? __fsub_rn(pv, cL.x) : CUDART_INF_F;
            float dR = R < n ? __fsub_rn(cR.x, pv) : CUDART_INF_F;
            while (true) {
                const bool right = dR < dL;
                const float da = right ? dR : dL;
                if (!(da < top[KMAX - 1])) break;
                const float oj = right ? cR.y : cL.y;
                const float d = fmaxf(da, fabsf(__fsub_rn(ov, oj)));
                if (d < top[KMAX - 1]) topk_insert<KMAX>(top, d);
                if (right) {
                    ++R;
                    if (R < n) {
                        cR = W[R];
                        dR = __fsub_rn(cR.x, pv);
                    } else {
                        dR = CUDART_INF_F;
                    }
                } else {
                    --L;
                    if (L >= 0) {
                        cL = W[L];
                        dL = __fsub_rn(pv, cL.x);
                    } else {
                        dL = CUDART_INF_F;
                    }
                }
            }
            const float eps = top[KMAX - 1];
            // walk axis: trim the visited window (L, R) to axis distance < eps
            while (L + 1 < s && !(__fsub_rn(pv, W[L + 1].x) < eps)) ++L;
            while (R - 1 > s && !(__fsub_rn(W[R - 1].x, pv) < eps)) --R;
            int c_walk = eps > 0.f ? R - L - 1 : 1;
            // other axis: [a, b) with a = first j with fl(ov - O[j].x) < eps,
            // b = first j with fl(O[j].x - ov) >= eps
            const int a = lower_search(0, n, [&](int j) { return __fsub_rn(ov, O[j].x) < eps; });
            const int b =
                lower_search(0, n, [&](int j) { return !(__fsub_rn(O[j].x, ov) < eps); });
            int c_oth = b - a;
            c_oth = c_oth < 1 ? 1 : c_oth;
            const int cx = on_y ? c_oth : c_walk;
            const int cy = on_y ? c_walk : c_oth;
            acc += psi[cx] + psi[cy];
            if (nx_out) {
                const int orig = perm_a[ra + ti];
                nx_out[t * n + orig] = cx;
                ny_out[t * n + orig] = cy;
                if (eps_out) eps_out[t * n + orig] = eps;
            }
        }
        acc = warp_sum_i64(acc);
        if (lane == 0) out[t] = (float)(psi_nk - ((double)acc / kFixScale) / (double)n);
        __syncwarp();
    }
}

template <int KMAX>
static cudaError_t ksg_launch(const Field& fa, const Field& fb, int k, const int64_t* psi_fix,
                              double psi_nk, const uint32_t* pa, const uint32_t* pb, int64_t N,
                              float* out, int32_t* nx, int32_t* ny, float* eps, int* status,
                              cudaStream_t st) {
    const int psi_len = (fa.n + 2) & ~1;
    const size_t smem = psi_len * sizeof(long long) + kKsgWarps * ksg_warp_bytes(fa.n_pad);
    if (smem > 48 * 1024) {
        cudaError_t e = cudaFuncSetAttribute(k_ksg_pairs<KMAX>,
                                             cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             (int)smem);
        if (e != cudaSuccess) return e;
    }
    int dev = 0, sms = 148;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    int64_t blocks = (N + kKsgWarps - 1) / kKsgWarps;
    blocks = blocks < (int64_t)sms * 16 ? blocks : (int64_t)sms * 16;
    note_launch();
    k_ksg_pairs<KMAX><<<(unsigned)blocks, kKsgWarps * 32, smem, st>>>(
        fa.sorted.as<float>(), fa.perm.as<uint16_t>(), fa.vals.as<float>(), fa.P,
        fb.sorted.as<float>(), fb.perm.as<uint16_t>(), fb.vals.as<float>(), fb.P, fa.n, fa.n_pad,
        k, (const long long*)psi_fix, psi_nk, pa, pb, N, out, nx, ny, eps, status);
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
