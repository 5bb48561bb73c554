// Internal types and helpers of the ccorr library (not part of the C ABI).
#pragma once

#include <cuda_runtime.h>
#include <math_constants.h>
#include <stdint.h>

#include <map>
#include <memory>
#include <string>
#include <vector>

#include "../../include/ccorr.h"

namespace cc {

// Device status word values written by kernels (first error wins).
enum : int { DEV_OK = 0, DEV_BAD_INDEX = 1, DEV_NONFINITE = 2, DEV_TIMEOUT = 3 };

// Fixed-point scale for order-independent sums of digamma and c*ln(c) terms:
// each table entry is round(value * 2^40) as int64.
constexpr double kFixScale = 1099511627776.0;  // 2^40

struct DevMem {
    void* p = nullptr;
    size_t bytes = 0;
    DevMem() = default;
    DevMem(const DevMem&) = delete;
    DevMem& operator=(const DevMem&) = delete;
    ~DevMem() {
        if (p) cudaFree(p);
    }
    cudaError_t alloc(size_t n) {
        if (p) cudaFree(p);
        p = nullptr;
        bytes = 0;
        if (n == 0) return cudaSuccess;
        cudaError_t e = cudaMalloc(&p, n);
        if (e == cudaSuccess) bytes = n;
        else p = nullptr;
        return e;
    }
    // Grow-only reallocation (contents are not kept).
    cudaError_t ensure(size_t n) { return n <= bytes ? cudaSuccess : alloc(n); }
    template <class T>
    T* as() const {
        return static_cast<T*>(p);
    }
};

// Pinned host memory, grow-only (device-to-host copies of small results
// land here asynchronously and are copied out after one stream wait).
struct HostMem {
    void* p = nullptr;
    size_t bytes = 0;
    HostMem() = default;
    HostMem(const HostMem&) = delete;
    HostMem& operator=(const HostMem&) = delete;
    ~HostMem() {
        if (p) cudaFreeHost(p);
    }
    cudaError_t ensure(size_t n) {
        if (n <= bytes) return cudaSuccess;
        if (p) cudaFreeHost(p);
        p = nullptr;
        bytes = 0;
        cudaError_t e = cudaMallocHost(&p, n);
        if (e == cudaSuccess) bytes = n;
        else p = nullptr;
        return e;
    }
    template <class T>
    T* as() const {
        return static_cast<T*>(p);
    }
};

// Per-point planes of one field, point-major [P][n_pad].
struct Field {
    int X = 0, Y = 0, Z = 0, n = 0, n_pad = 0;
    int64_t P = 0;
    DevMem vals;    // float    member values in member order
    DevMem sorted;  // float    ascending values (+inf padding)
    DevMem perm;    // uint16   stable argsort: sorted[t] = vals[perm[t]]
    DevMem rank2;   // int16    doubled average rank (1-based)
    DevMem zhat;    // float    (v - mean) / sqrt(sum of squared deviations)
    DevMem rhat;    // float    centred doubled ranks, unit norm
    DevMem mean;    // double   [P]
    DevMem ss;      // double   [P] sum of squared deviations
    std::map<int, std::unique_ptr<DevMem>> bins;   // B -> uint8 [P][n_pad]
    std::map<int, std::unique_ptr<DevMem>> hmarg;  // B -> int64 [P] fixed-point sum c ln c
    std::map<int, uint64_t> bins_version;          // B -> version the bins were built from
    uint64_t version = 0;                          // bumped by every value update
    DevMem staging;                                // host-update staging [n][P]
};

// A box of one field, with its point list and lazily built member-major
// compact planes ([nk][np_pad]) for the all-pairs contraction.
struct Region {
    int field = -1;
    cc_box box{};
    int64_t np = 0;
    std::vector<uint32_t> pts_host;
    DevMem pts;  // uint32 [np]
    int nk = 0;
    int64_t np_pad = 0;
    DevMem zT;  // float [nk][np_pad]
    DevMem rT;  // float [nk][np_pad]
    uint64_t planes_version = ~0ull;  // field version the planes were built from
    // reduced-precision K-major planes [rows_pad][kbytes] for the tensor-core
    // contraction, keyed by (plane: 0 zhat / 1 rhat) * 2 + fp8
    struct QPlane {
        DevMem q, inv, emax;
        int64_t rows_pad = 0;
        int kbytes = 0;
        uint64_t version = ~0ull;
    };
    std::map<int, std::unique_ptr<QPlane>> qplanes;
};

struct Partial {  // per-CTA extremes, reduced by a finishing kernel
    float max, min;
    unsigned long long argmax, argmin, count;
};

}  // namespace cc

struct cc_ctx {
    int device = 0;
    cudaStream_t stream = nullptr;
    bool own_stream = false;
    std::string err;
    std::vector<std::unique_ptr<cc::Field>> fields;
    std::vector<std::unique_ptr<cc::Region>> regions;
    cc::DevMem status;  // int device status word
    // scratch
    cc::DevMem pair_a, pair_b, vals_out, partials, rp_out, ksg_nx, ksg_ny, ksg_eps, mixed;
    cc::DevMem approx;  // chunk extremes exported by cc_all_pairs_approx
    cc::HostMem host_out;  // pinned landing area of cc_all_pairs_topk's results
    // surrogate training: pinned epoch permutations (the next one is drawn
    // while an epoch runs) and the periodic loss reads
    cc::HostMem sur_order[2], sur_loss;
    std::map<int, std::unique_ptr<cc::DevMem>> psi_fix;   // n -> int64 [n+1]
    std::map<int, std::unique_ptr<cc::DevMem>> clogc_fix; // n -> int64 [n+1]
    // host-to-device copies of an update overlap its ingest: a second stream
    // and one event per chunk (created on first use)
    cudaStream_t copy_stream = nullptr;
    std::vector<cudaEvent_t> copy_events;
    // captured launch sequences of cc_all_pairs_topk, keyed by every buffer
    // address and size they use
    struct CachedGraph {
        std::vector<uint64_t> key;
        cudaGraphExec_t exec;
        int kernels;
    };
    std::vector<CachedGraph> topk_graphs;
    ~cc_ctx() {
        for (auto& g : topk_graphs) cudaGraphExecDestroy(g.exec);
        for (cudaEvent_t e : copy_events) cudaEventDestroy(e);
        if (copy_stream) cudaStreamDestroy(copy_stream);
    }
};

namespace cc {

// Counts kernel launches of the library (cc_launch_count).
void note_launch(int kernels = 1);

// Streaming multiprocessors of the current device (grid sizes scale with it).
int sm_count();

// Raise a kernel's dynamic shared-memory limit on the current device to at
// least `bytes`, never lowering it: launches captured into a CUDA graph keep
// their own sizes, so a later call with a smaller size must leave the limit
// where an earlier capture needs it.
template <class Kernel>
cudaError_t raise_smem_limit(Kernel* kernel, size_t bytes) {
    cudaFuncAttributes a{};
    cudaError_t e = cudaFuncGetAttributes(&a, kernel);
    if (e != cudaSuccess) return e;
    if ((size_t)a.maxDynamicSharedSizeBytes >= bytes) return cudaSuccess;
    return cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
}

// Kernel launchers (defined in the .cu files), all on `st`.
// in: member-major [n][in_stride] (P points used), vals: point-major [P][n_pad]
cudaError_t launch_ingest(const float* in, int n, int64_t P, int64_t in_stride, int n_pad,
                          float* vals, int* status, cudaStream_t st);
// bin planes rebuilt inside the per-point pass (at most two bin counts)
struct PrepBins {
    int count = 0;
    int B[2] = {0, 0};
    uint8_t* bins[2] = {nullptr, nullptr};
    long long* hmarg[2] = {nullptr, nullptr};
    const long long* clogc = nullptr;
};
cudaError_t launch_aggregate(const Field& f, int bx, int by, int bz, int Xc, int Yc, int64_t Pc,
                             int mode, float* out, cudaStream_t st);
// per-point planes of points [p_begin, p_end) (p_end < 0: all points)
cudaError_t launch_point_prep(const Field& f, cudaStream_t st, const PrepBins& pb = PrepBins(),
                              int64_t p_begin = 0, int64_t p_end = -1);
cudaError_t launch_bins(const Field& f, int B, const int64_t* clogc_fix, uint8_t* bins,
                        int64_t* hmarg, cudaStream_t st);
cudaError_t launch_region_planes(const Field& f, const Region& r, cudaStream_t st);

cudaError_t launch_pearson_pairs(const float* plane_a, int64_t Pa, const float* plane_b,
                                 int64_t Pb, int n_pad, const uint32_t* pa, const uint32_t* pb,
                                 int64_t N, float* out, int* status, cudaStream_t st);
cudaError_t launch_hist_pairs(const uint8_t* bins_a, const int64_t* hm_a, int64_t Pa,
                              const uint8_t* bins_b, const int64_t* hm_b, int64_t Pb, int n,
                              int n_pad, int B, const int64_t* clogc_fix, const uint32_t* pa,
                              const uint32_t* pb, int64_t N, float* out, int* status,
                              cudaStream_t st);
cudaError_t launch_ksg_pairs(const Field& fa, const Field& fb, int k, const int64_t* psi_fix,
                             const uint32_t* pa, const uint32_t* pb, int64_t N, float* out,
                             int32_t* nx, int32_t* ny, float* eps, int* status, cudaStream_t st);
cudaError_t launch_sample_lds(int kind, const int* ext, const double* alpha, int self,
                              const uint32_t* pts_a, const uint32_t* pts_b, uint64_t first,
                              int64_t N, uint32_t* pa, uint32_t* pb, cudaStream_t st);
cudaError_t launch_sample_pairs(const uint32_t* pts_a, int64_t na, const uint32_t* pts_b,
                                int64_t nb, int self, uint64_t seed, uint64_t stream,
                                uint64_t first, int64_t N, uint32_t* pa, uint32_t* pb,
                                cudaStream_t st);
constexpr int64_t kSegChunk = 8192;  // values per CTA in the segment reduction
cudaError_t launch_segment_extremes(const float* values, const int64_t* chunk_bounds,
                                    int64_t n_chunks, const int64_t* seg_first_chunk, int n_seg,
                                    Partial* chunk_part, Partial* out, cudaStream_t st);
cudaError_t launch_allpairs_f32(const float* A, int64_t lda, const float* B, int64_t ldb, int nk,
                                int64_t PA, int64_t PB, int self, float* C, int64_t ldc,
                                Partial* partials, Partial* result, cudaStream_t st);
size_t allpairs_partials(int64_t PA, int64_t PB);

// reduced precision (tc_gemm.cu, mixed.cu)
// State of one histogram selection (keys >= threshold are candidates).
struct Select {
    unsigned prefix;     // top-12-bit bin found by the first pass
    unsigned need;       // keys still needed inside that bin
    unsigned threshold;  // order-preserving key threshold; 0 = every key
    unsigned count;      // compacted candidates
    unsigned overflow;   // candidates beyond capacity
    unsigned pass1;      // candidates of the first pass (the second appends after them)
};
// Device record of one extreme side of a certified all-pairs call, read back
// by the host once at the end.
struct SideState {
    Select sel;               // first and second pass counts, overflow, threshold
    unsigned pad;
    unsigned long long best;  // (key of best value, inverted pair index)
    float thr[2];             // second-pass threshold, bound
};
// C[m][n] = sum_k A[m sam + k sak] B[n sbn + k sbk] on the tensor cores
// (tc_mm.cu): BF16 (flag 1) or FP32 operands, N <= 256; with kc < K the z-th
// K slice writes part[z][M][N]; B's row b_ones (>= 0) reads as 1.
cudaError_t launch_tc_mm(const void* A, int a_bf16, int64_t sam, int64_t sak, const void* B,
                         int b_bf16, int64_t sbn, int64_t sbk, int64_t b_ones, float* C,
                         int64_t ldc, int M, int N, int64_t K, int64_t kc, float* part,
                         int* status, cudaStream_t st);
cudaError_t launch_sur_screen_tc(const float* Ea, const float* Ua, const float* Eb,
                                 const void* wb, const float* w, int64_t oW3, int64_t ow4,
                                 int64_t ob4, const uint32_t* pts_a, const uint32_t* pts_b,
                                 int64_t na, int64_t nb, int self, int X, int Y, int Z,
                                 float tmean, float tsd, float* pred, int* status,
                                 cudaStream_t st);
cudaError_t launch_tc_chunk_extremes(bool fp8, bool scaled, const void* qa, int64_t na,
                                     int64_t na_pad, const void* qb, int64_t nb, int64_t nb_pad, int64_t kbytes,
                                     int self, const float* inv_sa, const float* inv_sb,
                                     float* cmax, float* cmin, unsigned* hist0, int* status,
                                     cudaStream_t st);
cudaError_t launch_quantize(bool fp8, const float* plane, int n_pad, int n, const uint32_t* pts,
                            int64_t np, int64_t np_pad, int kbytes, void* q, float* inv_scale,
                            unsigned* emax_bits, cudaStream_t st);
cudaError_t launch_quantize_ranks(const int16_t* rank2, int n_pad, int n, const uint32_t* pts,
                                  int64_t np, int64_t np_pad, int kbytes, void* q,
                                  float* inv_scale, cudaStream_t st);
cudaError_t launch_select_top(const float* v, int64_t N, float sign, unsigned want,
                              unsigned* hist, Select* sel, uint32_t* out, unsigned cap,
                              cudaStream_t st, const unsigned* nchunks = nullptr);
// Both extreme sides at once: keys of +v0 (side 0) and -v1 (side 1); side s
// selects at least want_s chunk ids into out + s * cap using ss[s].sel; hist
// holds 2 x 4096 bins, zeroed, or with hist0_built the first-level (11-bit)
// histograms that launch_tc_chunk_extremes added.
cudaError_t launch_select_top2(const float* v0, const float* v1, int64_t N, unsigned want0,
                               unsigned want1, unsigned* hist, bool hist0_built, SideState* ss,
                               uint32_t* out, unsigned cap, cudaStream_t st);
// second compaction of both sides (keys in [thr_s, first threshold))
cudaError_t launch_compact_second2(const float* v0, const float* v1, int64_t N, SideState* ss,
                                   uint32_t* out, unsigned cap, cudaStream_t st);
// Dot2 refinement of the candidate chunks of both sides (first_pass: every
// id from 0, else the ids the second compaction appended); wide: a loose
// bound (FP8), more blocks per side.
cudaError_t launch_refine_chunks2(const float* plane_a, const float* plane_b, int n_pad, int n,
                                  const uint32_t* pts_a, int64_t na, const uint32_t* pts_b,
                                  int64_t nb, int self, int64_t na_pad, const uint32_t* ids,
                                  unsigned cap, SideState* ss, bool first_pass, float* vals,
                                  unsigned long long* pair_ids, bool wide, cudaStream_t st);
cudaError_t launch_second_threshold2(SideState* ss, const unsigned* emax_a,
                                     const unsigned* emax_b, float acc_rel, cudaStream_t st);
// top-k (<= 8192) of up to 8192 selected entries, sorted descending by value,
// then by smallest id; scratch holds 8192 64-bit keys
cudaError_t launch_sort_top(const float* vals, const unsigned long long* pids,
                            const uint32_t* sel_idx, const unsigned* count, unsigned cap,
                            float sign, int topk, float* out_vals, unsigned long long* out_ids,
                            unsigned long long* scratch, cudaStream_t st);
cudaError_t launch_sort_top_ids(const float* vals, const uint32_t* sel_idx, const unsigned* count,
                                unsigned cap, int topk, float* out_vals,
                                unsigned long long* out_ids, unsigned long long* scratch,
                                cudaStream_t st);
cudaError_t launch_dot2_pairs(const float* A, int64_t Pa, const float* B, int64_t Pb, int n_pad,
                              int n, const uint32_t* pa, const uint32_t* pb, int64_t N, float* out,
                              int* status, cudaStream_t st);

}  // namespace cc
