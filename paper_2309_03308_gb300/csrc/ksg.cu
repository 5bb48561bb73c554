// Kraskov (KSG) mutual information on a batch of point pairs (Section 3.2).
//
// For a pair (p, q) the joint samples are z_i = (x_i, y_i), x = members of
// p, y = members of q. With fp32 differences (bit-identical to the
// definition):
//   eps_i = k-th smallest d_ij = max(|x_i - x_j|, |y_i - y_j|) over j != i
//   n_x,i = 1 + #{j != i : |x_i - x_j| < eps_i}, n_y,i likewise
//   MI    = psi(n) + psi(k) - (1/n) sum_i [psi(n_x,i) + psi(n_y,i)]
//
// Design (one warp per group of pairs, one lane per sample i; the device
// steps are in ksg_dev.cuh):
//   For each pair the warp stages (x, y) in x-sorted order, (y, x) in
//   y-sorted order and each sample's y-sorted position in shared memory; the
//   per-point sorted values and argsorts come from ingest, so staging is
//   gathers only. The samples of the group's pairs form one stream that the
//   lanes take 32 at a time, so fewer lanes idle at the end of a pair.
//
//   eps_i: walk outward from i along ONE axis, over that axis's sorted order,
//   on both sides at once; every visited j offers d_ij. The first k
//   positions are taken unconditionally and sorted by a fixed network; the
//   first step offers the next four positions of each side, every later step
//   the next two (four again in the pair-batch form, whose walks are long),
//   to a sorted register list of the k smallest (the new values
//   sorted, folded into the list's top entries, bitonic merger) and passes
//   the positions whose axis distance was below the list's k-th value. When
//   both next axis distances are not below the k-th value no unvisited j can
//   enter, so the walk stops with the exact k-th smallest. The walk length is
//   about the number of samples within eps_i along the axis, so each lane
//   walks along the axis on which the ~0.8 sqrt(k n) sorted positions nearest
//   to the sample span the wider range. Sentinels (+-inf) around the staged arrays
//   keep the step free of bounds checks, and all lanes run the same code on
//   lane-selected arrays.
//
//   Counts: the walk's final window holds every j with axis distance below
//   eps_i (trimmed at its ends); the other axis is counted with two binary
//   searches on its sorted values (fl32 differences are monotone, so the set
//   is a contiguous range). The self sample is in the range exactly when
//   eps_i > 0, giving 1 + #{j != i} as defined.
//
//   The digamma sum uses a fixed-point table (2^-40), exact and order
//   independent; psi(n) + psi(k) and the final scaling are FP64.
#include "internal.cuh"
#include "ksg_dev.cuh"

namespace cc {

double digamma_int_host(int m);

constexpr int kKsgWarps = 8;
// The pair-batch form holds one staged pair per warp in shared memory; for
// large n the slot, not the register file, limits the warps an SM can run,
// so a block takes as many warps as leave room for two blocks per SM.
constexpr int kMaxPairWarps = 16;
constexpr int kMaxGroup = 4;

template <int KMAX>
__global__ void __launch_bounds__(kMaxPairWarps * 32)
    k_ksg_pairs(const float* __restrict__ sorted_a, const uint16_t* __restrict__ perm_a,
                const float* __restrict__ vals_a, int64_t Pa, const float* __restrict__ sorted_b,
                const uint16_t* __restrict__ perm_b, const float* __restrict__ vals_b, int64_t Pb,
                int n, int n_pad, int k, int G, int team, const long long* __restrict__ psi_fix,
                double psi_nk, double fix_over_n, const uint32_t* __restrict__ pa,
                const uint32_t* __restrict__ pb, int64_t N, float* __restrict__ out,
                int32_t* __restrict__ nx_out,
                int32_t* __restrict__ ny_out, float* __restrict__ eps_out, int* status) {
    extern __shared__ __align__(16) unsigned char ksg_smem[];
    __shared__ long long team_part[kMaxPairWarps][kMaxGroup];
    long long* psi = reinterpret_cast<long long*>(ksg_smem);
    const int psi_len = (n + 2) & ~1;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    // `team` consecutive warps share one staged group of pairs and split its
    // samples; the first warp of a team stages and writes the results
    const int team_id = warp / team, tw = warp % team, tl = tw * 32 + lane;
    const int teams = (blockDim.x >> 5) / team;
    const size_t slot_bytes = ksg_slot_bytes(n_pad, KMAX);
    unsigned char* wbase =
        ksg_smem + psi_len * sizeof(long long) + (size_t)team_id * G * slot_bytes;
    auto team_sync = [&]() {
        if (team == 1) __syncwarp();
        else asm volatile("bar.sync %0, %1;" ::"r"(1 + team_id), "r"(team * 32) : "memory");
    };
    for (int i = threadIdx.x; i <= n; i += blockDim.x) psi[i] = psi_fix[i];
    __syncthreads();

    const int64_t ngroups = (N + G - 1) / G;
    for (int64_t g = (int64_t)blockIdx.x * teams + team_id; g < ngroups;
         g += (int64_t)gridDim.x * teams) {
        const int64_t t0 = g * G;
        const int gc = (int)min((int64_t)G, N - t0);
        unsigned valid = 0;
        for (int sl = 0; sl < gc; ++sl) {
            const uint32_t p = pa[t0 + sl], q = pb[t0 + sl];
            if (p >= Pa || q >= Pb) {
                if (tl == 0) {
                    out[t0 + sl] = CUDART_NAN_F;
                    set_status(status, DEV_BAD_INDEX);
                }
                continue;
            }
            valid |= 1u << sl;
            const int64_t ra = (int64_t)p * n_pad, rb = (int64_t)q * n_pad;
            if (tw == 0)
                ksg_stage<KMAX>(wbase + sl * slot_bytes, n, n_pad, sorted_a + ra, perm_a + ra,
                                vals_a + ra, sorted_b + rb, perm_b + rb, vals_b + rb);
        }
        team_sync();  // the staged slots are visible to the whole team

        long long acc[kMaxGroup];
#pragma unroll
        for (int u = 0; u < kMaxGroup; ++u) acc[u] = 0;
        const int items = gc * n;
        for (int it = tl; it < items; it += team * 32) {
            const int sl = it / n, ti = it - sl * n;
            if (!((valid >> sl) & 1u)) continue;
            int cx, cy;
            float eps;
            // pair-batch form (n > 256 or n < 32): long walks take eight
            // positions in every step
            const long long v = ksg_sample<KMAX, true>(wbase + sl * slot_bytes, n, n_pad, k, ti,
                                                       psi, nx_out ? &cx : nullptr, &cy, &eps);
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
                if (lane == 0) team_part[warp][u] = sum;
            }
        }
        // every warp of the team is done with the slots and its part is stored
        team_sync();
        if (tw == 0 && lane == 0) {
            for (int u = 0; u < gc; ++u) {
                long long sum = 0;
                for (int w = 0; w < team; ++w) sum += team_part[warp + w][u];
                if ((valid >> u) & 1u) out[t0 + u] = (float)(psi_nk - (double)sum * fix_over_n);
            }
        }
        // the parts are read before the team's next group overwrites them
        team_sync();
    }
}

// Sample-stream form for 32 <= n <= 256: warp w owns the contiguous pairs
// [w P_w, (w + 1) P_w) and walks their samples as one stream, 32 per round
// (lane l takes stream position 32 r + l), so no lane idles at the end of a
// pair. A round spans at most two pairs, so two slots per warp suffice: pair
// p is staged into slot p & 1 before the first round that reaches it, and
// its slot is reused for pair p + 2, whose first sample lies more than 32
// positions after p's last. At most one pair ends per round; its digamma sum
// is reduced over the warp and written at the end of that round.
template <int KMAX>
__global__ void __launch_bounds__(kKsgWarps * 32)
    k_ksg_stream(const float* __restrict__ sorted_a, const uint16_t* __restrict__ perm_a,
                 const float* __restrict__ vals_a, int64_t Pa, const float* __restrict__ sorted_b,
                 const uint16_t* __restrict__ perm_b, const float* __restrict__ vals_b, int64_t Pb,
                 int n, int n_pad, int k, int64_t per_warp, const long long* __restrict__ psi_fix,
                 double psi_nk, double fix_over_n, const uint32_t* __restrict__ pa,
                 const uint32_t* __restrict__ pb, int64_t N, float* __restrict__ out,
                 int32_t* __restrict__ nx_out, int32_t* __restrict__ ny_out,
                 float* __restrict__ eps_out, int* status) {
    extern __shared__ __align__(16) unsigned char ksg_smem[];
    long long* psi = reinterpret_cast<long long*>(ksg_smem);
    const int psi_len = (n + 2) & ~1;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const size_t slot_bytes = ksg_slot_bytes(n_pad, KMAX);
    unsigned char* wbase = ksg_smem + psi_len * sizeof(long long) + (size_t)warp * 2 * slot_bytes;
    for (int i = threadIdx.x; i <= n; i += blockDim.x) psi[i] = psi_fix[i];
    __syncthreads();

    const int64_t p0 = ((int64_t)blockIdx.x * kKsgWarps + warp) * per_warp;
    const int64_t p1 = min(N, p0 + per_warp);
    if (p0 >= p1) return;
    // the round's first stream position as (pair tr, sample tir); positions
    // advance by 32 per round and n >= 32, so a round crosses at most one
    // pair boundary and no division is needed
    int64_t tr = p0;
    int tir = 0;
    int64_t staged = p0;  // next pair to stage
    unsigned valid = 0;   // bit (p & 1): pair in that slot is valid
    long long acc[2] = {0, 0};
    while (tr < p1) {
        const int64_t t_last = min(p1 - 1, tr + (tir + 31 >= n ? 1 : 0));
        for (; staged <= t_last; ++staged) {  // warp-uniform
            const int sl = (int)(staged & 1);
            const uint32_t p = pa[staged], q = pb[staged];
            if (p < Pa && q < Pb) {
                valid |= 1u << sl;
                const int64_t ra = (int64_t)p * n_pad, rb = (int64_t)q * n_pad;
                ksg_stage<KMAX>(wbase + sl * slot_bytes, n, n_pad, sorted_a + ra, perm_a + ra,
                                vals_a + ra, sorted_b + rb, perm_b + rb, vals_b + rb);
            } else {
                valid &= ~(1u << sl);
                if (lane == 0) {
                    out[staged] = CUDART_NAN_F;
                    set_status(status, DEV_BAD_INDEX);
                }
            }
        }
        int ti = tir + lane;
        int64_t t = tr;
        if (ti >= n) {
            ti -= n;
            ++t;
        }
        const int sl = (int)(t & 1);
        if (t < p1 && ((valid >> sl) & 1u)) {
            int cx, cy;
            float eps;
            const long long v = ksg_sample<KMAX>(wbase + sl * slot_bytes, n, n_pad, k, ti, psi,
                                                 nx_out ? &cx : nullptr, &cy, &eps);
            if (sl) acc[1] += v;
            else acc[0] += v;
            if (nx_out) {
                const int orig = perm_a[(int64_t)pa[t] * n_pad + ti];
                nx_out[t * n + orig] = cx;
                ny_out[t * n + orig] = cy;
                if (eps_out) eps_out[t * n + orig] = eps;
            }
        }
        // pair tr ends in this round when its last sample n - 1 <= tir + 31
        if (tir + 32 >= n) {
            const int se = (int)(tr & 1);
            const long long sum = warp_sum_i64(se ? acc[1] : acc[0]);
            if (lane == 0 && ((valid >> se) & 1u))
                out[tr] = (float)(psi_nk - (double)sum * fix_over_n);
            if (se) acc[1] = 0;
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

template <int KMAX>
static cudaError_t ksg_launch(const Field& fa, const Field& fb, int k, const int64_t* psi_fix,
                              double psi_nk, const uint32_t* pa, const uint32_t* pb, int64_t N,
                              float* out, int32_t* nx, int32_t* ny, float* eps, int* status,
                              cudaStream_t st) {
    // two pairs per warp while n is small, so the sample stream fills the lanes
    // (more pairs per warp costs occupancy through shared memory)
    const int G = fa.n_pad <= 128 ? 2 : 1;
    // for large n two (n_pad 512) or four (n_pad 1024) warps share one staged
    // pair, which divides the shared memory per warp (the slot, not the
    // register file, limits the warps)
    const int team = fa.n_pad >= 1024 ? 4 : (fa.n_pad >= 512 ? 2 : 1);
    const int psi_len = (fa.n + 2) & ~1;
    int dev = 0, sms = 148, smem_sm = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    cudaDeviceGetAttribute(&smem_sm, cudaDevAttrMaxSharedMemoryPerMultiprocessor, dev);
    // pair-batch form: as many warps per block as leave room for two blocks
    // per SM (1 KB per block is reserved by the runtime)
    const size_t slot = (size_t)G * ksg_slot_bytes(fa.n_pad, KMAX);
    const size_t psi_b = psi_len * sizeof(long long);
    const size_t smem_free = (size_t)smem_sm / 2 - 1024 - psi_b -
                             sizeof(long long) * kMaxPairWarps * kMaxGroup;
    int pw = team * (int)(smem_free / slot);
    static const int regs = [] {  // and two blocks' registers
        cudaFuncAttributes fa_attr{};
        return cudaFuncGetAttributes(&fa_attr, k_ksg_pairs<KMAX>) == cudaSuccess
                   ? fa_attr.numRegs : 64;
    }();
    pw = std::min(pw, 65536 / (2 * 32 * std::max(regs, 1)));
    pw = pw < team ? team : (pw > kMaxPairWarps ? kMaxPairWarps : pw);
    pw -= pw % team;
    const size_t smem = psi_b + (size_t)(pw / team) * slot;
    if (smem > 48 * 1024) {
        cudaError_t e = cudaFuncSetAttribute(k_ksg_pairs<KMAX>,
                                             cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             (int)smem);
        if (e != cudaSuccess) return e;
    }
    if (fa.n >= 32 && fa.n_pad <= 256) {  // sample stream, two slots per warp
        const size_t smem2 =
            psi_len * sizeof(long long) + kKsgWarps * 2 * ksg_slot_bytes(fa.n_pad, KMAX);
        if (smem2 > 48 * 1024) {
            cudaError_t e = cudaFuncSetAttribute(k_ksg_stream<KMAX>,
                                                 cudaFuncAttributeMaxDynamicSharedMemorySize,
                                                 (int)smem2);
            if (e != cudaSuccess) return e;
        }
        // about 32 blocks' worth of warps per SM, so the last pairs spread thinly
        const int64_t want_warps = (int64_t)sms * 32 * kKsgWarps;
        const int64_t per_warp = (N + want_warps - 1) / want_warps;
        const int64_t warps = (N + per_warp - 1) / per_warp;
        const int64_t blocks = (warps + kKsgWarps - 1) / kKsgWarps;
        note_launch();
        k_ksg_stream<KMAX><<<(unsigned)blocks, kKsgWarps * 32, smem2, st>>>(
            fa.sorted.as<float>(), fa.perm.as<uint16_t>(), fa.vals.as<float>(), fa.P,
            fb.sorted.as<float>(), fb.perm.as<uint16_t>(), fb.vals.as<float>(), fb.P, fa.n,
            fa.n_pad, k, per_warp, (const long long*)psi_fix, psi_nk, 1.0 / (kFixScale * fa.n),
            pa, pb, N, out, nx, ny, eps, status);
        return cudaGetLastError();
    }
    const int64_t groups = (N + G - 1) / G;
    int64_t blocks = (groups + pw / team - 1) / (pw / team);
    blocks = blocks < (int64_t)sms * 16 ? blocks : (int64_t)sms * 16;
    note_launch();
    k_ksg_pairs<KMAX><<<(unsigned)blocks, pw * 32, smem, st>>>(
        fa.sorted.as<float>(), fa.perm.as<uint16_t>(), fa.vals.as<float>(), fa.P,
        fb.sorted.as<float>(), fb.perm.as<uint16_t>(), fb.vals.as<float>(), fb.P, fa.n, fa.n_pad,
        k, G, team, (const long long*)psi_fix, psi_nk, 1.0 / (kFixScale * fa.n), pa, pb, N, out,
        nx, ny, eps, status);
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
    if (k <= 4) CC_KSG(4);
    if (k <= 8) CC_KSG(8);
    if (k <= 10) CC_KSG(10);
    if (k <= 16) CC_KSG(16);
    CC_KSG(32);
#undef CC_KSG
}

}  // namespace cc
