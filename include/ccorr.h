/*
 * ccorr -- point-to-point correlation measures between ensemble member
 * vectors at pairs of 3D grid points, on one GB300 GPU (sm_103a).
 *
 * Method: arxiv 2309.03308, "Adaptive Sampling of 3D Spatial Correlations for
 * Focus+Context Visualization". The library evaluates Pearson (PPMCC),
 * Spearman, joint-histogram mutual information and the Kraskov (KSG) k-NN
 * mutual-information estimator (Section 3.2) on batches of point pairs, all
 * pairs between two regions ("bricks", Section 3), and reduces them to the
 * per-region-pair maximum (Section 3: the brick-pair indicator).
 *
 * Conventions shared by every entry point
 *   - Every function returns cc_status (0 = CC_OK, negative = error) and never
 *     throws or aborts across the ABI. cc_last_error() gives a message.
 *   - Work is queued on the context's CUDA stream. Functions that return data
 *     in HOST memory synchronise that stream before they return; functions
 *     writing only DEVICE memory are asynchronous. cc_sync() waits and reports
 *     any error a kernel recorded in the context's device status word.
 *   - Caller buffers stay owned by the caller. Flags named *_is_device / *_on_device
 *     say whether a pointer is device memory (e.g. a PyTorch CUDA tensor's
 *     data pointer) or host memory.
 *   - A field is an ensemble on an X x Y x Z grid with n members, fp32, given
 *     in layout [n][Z][Y][X] (member-major, x fastest). Grid point ids are
 *     linear: id = x + X * (y + Y * z).
 *   - Regions are half-open axis-aligned boxes of one field. The points of a
 *     region are enumerated x fastest, then y, then z; a region-local index
 *     is a position in that enumeration.
 *   - Measures with identical results on both GPUs are bit-exact: average
 *     ranks, bin ids and KSG neighbour counts (from the same fp32 input).
 *   - One context may be used by one host thread at a time.
 */
#ifndef CCORR_H
#define CCORR_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct cc_ctx cc_ctx;
typedef int32_t cc_status;

#define CC_OK 0
#define CC_ERR_INVALID_ARG (-1)  /* bad pointer, size, id or parameter */
#define CC_ERR_OOM (-2)          /* device or host allocation failed */
#define CC_ERR_CUDA (-3)         /* a CUDA call failed (message has the CUDA error) */
#define CC_ERR_NONFINITE (-4)    /* NaN or Inf in a loaded field */
#define CC_ERR_TIMEOUT (-5)      /* a bounded device-side wait gave up */
#define CC_ERR_UNSUPPORTED (-6)  /* valid request the library or device cannot run */

/* Measures (Section 3.2; Spearman is a project addition). */
#define CC_PEARSON 0   /* PPMCC of the member vectors */
#define CC_SPEARMAN 1  /* PPMCC of the average (tie-averaged) ranks */
#define CC_MI_BINNED 2 /* MI of the joint histogram, bins equal-width over each point's [min,max] */
#define CC_MI_KSG 3    /* Kraskov estimator, Chebyshev k-NN in the joint space */

/* Arithmetic of Pearson/Spearman (other measures ignore it). */
#define CC_FP32 0       /* fp32 values and accumulation */
#define CC_BF16 1       /* bf16 tensor-core contraction, fp32 accumulation */
#define CC_FP8_E4M3 2   /* fp8 e4m3 (per-point scale) tensor-core contraction, fp32 accumulation */
#define CC_FP32_DOT2 3  /* compensated fp32 (Dot2: TwoProduct/TwoSum) */

/*
 * Measure parameters.
 *   measure   CC_PEARSON .. CC_MI_KSG
 *   k         KSG neighbour count, 1 <= k <= min(n-1, 32); k = -1 selects the
 *             paper's rule k = ceil(3n/100) (Section 3.2). Ignored otherwise.
 *   bins      histogram bins per variable for CC_MI_BINNED, 2..16.
 *   precision CC_FP32 .. CC_FP32_DOT2 (Pearson/Spearman only).
 *   flags     reserved, must be 0.
 */
typedef struct {
    int32_t measure;
    int32_t k;
    int32_t bins;
    int32_t precision;
    int32_t flags;
} cc_params;

/* Half-open voxel box [x0,x1) x [y0,y1) x [z0,z1). */
typedef struct {
    int32_t x0, y0, z0, x1, y1, z1;
} cc_box;

/*
 * Extremes of one region pair (Section 3: maximum over point pairs; Section
 * 5.3 also uses the minimum). argmax/argmin are pair indices whose meaning is
 * given by the producing call; ties resolve to the smallest index. count is
 * the number of pairs reduced; with count == 0, max = -inf and min = +inf.
 */
typedef struct {
    float max;
    float min;
    uint64_t argmax;
    uint64_t argmin;
    uint64_t count;
} cc_rp_result;

/* ------------------------------------------------------------------------ context */

/*
 * Create a context on CUDA device `device`. `stream` is a cudaStream_t to
 * queue work on (e.g. a PyTorch stream handle) or NULL for a stream the
 * context creates and owns. *out receives the context.
 */
cc_status cc_create(int device, void* stream, cc_ctx** out);

/* Release every device buffer of the context (fields, regions, scratch). */
cc_status cc_destroy(cc_ctx* ctx);

/* Message of the last failing call on this context; owned by the context. */
const char* cc_last_error(const cc_ctx* ctx);

/* Wait for the context's stream; returns a device-recorded error if any. */
cc_status cc_sync(cc_ctx* ctx);

/* --------------------------------------------------------------- field ingest */

/*
 * Load an ensemble field and precompute its per-point planes (Section 3: an
 * ensemble of n members on an X x Y x Z grid; Section 3.2: PPMCC needs only
 * the means and variances). data is fp32 [n][Z][Y][X]; data_is_device says
 * where it lives. The library copies it; the caller keeps ownership.
 * Per grid point the library computes, on the GPU: FP64 mean and sum of
 * squared deviations, the unit-norm centred vector used by Pearson, the
 * doubled average ranks and unit-norm centred ranks used by Spearman, the
 * member values in ascending order with their stable argsort (KSG).
 * Requires 2 <= n <= 1024. A NaN or Inf anywhere returns CC_ERR_NONFINITE and
 * loads nothing. *field_id receives the new field's id.
 */
cc_status cc_load_field(cc_ctx* ctx, const float* data, int data_is_device, int X, int Y, int Z,
                        int n, int32_t* field_id);

/*
 * Replace the member values of an already loaded field (same X, Y, Z, n) and
 * recompute every per-point plane in place, reusing the field's buffers (an
 * update from host memory stages through a device buffer of the field's size,
 * allocated on the first such call and kept with the field). Planes of the
 * field's regions and bin planes are rebuilt on their next use. Asynchronous:
 * a NaN or Inf is reported as CC_ERR_NONFINITE by cc_sync or by the next call
 * that returns host data. From host memory of 64 MB or more the copy runs in
 * eight point ranges on a second stream of the context, each range's planes
 * computed on the context's stream as soon as it has arrived; the host
 * buffer must stay unchanged until the context's stream reaches this call's
 * work (page-locked memory makes the copy asynchronous).
 */
cc_status cc_update_field(cc_ctx* ctx, int32_t field_id, const float* data, int data_is_device);

/*
 * Spatial aggregate of a field (Section 3.3: mean-tree / max-tree levels that
 * let sampling run on a coarser copy when the full ensemble does not fit):
 * blocks of bx x by x bz grid points (the last block of an axis is smaller
 * when the extent is not a multiple) become one grid point of a new field of
 * ceil(X/bx) x ceil(Y/by) x ceil(Z/bz) points with the same n members. Per
 * block and member: CC_AGG_MEAN the mean (FP64 sum of the block's fp32
 * values divided by its point count, rounded to fp32), CC_AGG_MAX the
 * maximum. The new field (with all its planes) is returned in *out_field_id.
 */
#define CC_AGG_MEAN 0
#define CC_AGG_MAX 1
cc_status cc_aggregate_field(cc_ctx* ctx, int32_t field_id, int bx, int by, int bz, int mode,
                             int32_t* out_field_id);

/* Drop a field and its regions' device planes. */
cc_status cc_free_field(cc_ctx* ctx, int32_t field_id);

/*
 * Read back per-point planes for inspection (bit-exact tests). plane:
 *   CC_PLANE_RANK2   int32 [count][n]  doubled average rank 2*rank (1-based)
 *   CC_PLANE_BINS    uint8 [count][n]  bin ids for `bins` bins
 *   CC_PLANE_SORTED  float [count][n]  ascending member values
 *   CC_PLANE_ZHAT    float [count][n]  (v - mean) / sqrt(sum of squared deviations)
 * pts are `count` grid point ids (host); out is host memory.
 */
#define CC_PLANE_RANK2 0
#define CC_PLANE_BINS 1
#define CC_PLANE_SORTED 2
#define CC_PLANE_ZHAT 3
cc_status cc_get_plane(cc_ctx* ctx, int32_t field_id, int plane, int bins, const uint32_t* pts,
                       int64_t count, void* out);

/* --------------------------------------------------------------------- regions */

/*
 * Define `count` regions (bricks, Section 3) of field `field_id` from boxes
 * (host array). region_ids (host, `count` entries) receives their ids.
 */
cc_status cc_define_regions(cc_ctx* ctx, int32_t field_id, const cc_box* boxes, int count,
                            int32_t* region_ids);

/*
 * Partition the field into axis-aligned boxes of bx x by x bz voxels
 * (Section 3: bricks; boxes at the high boundary are smaller when the grid
 * size is not a multiple). Boxes are enumerated x fastest, then y, then z.
 * Up to `cap` ids go to region_ids; *count receives the number of regions.
 * Returns CC_ERR_INVALID_ARG (and defines nothing) if cap is too small.
 */
cc_status cc_partition_regular(cc_ctx* ctx, int32_t field_id, int bx, int by, int bz,
                               int32_t* region_ids, int cap, int* count);

/* Number of points of a region (*npoints) and its box (*box, may be NULL). */
cc_status cc_region_info(cc_ctx* ctx, int32_t region_id, int64_t* npoints, cc_box* box);

/* ------------------------------------------------------------------- sampling */

/*
 * Uniform random point pairs between two regions (Section 3.1: random
 * samples in the 6D space of a brick pair). Pair t uses one Philox4x64-10
 * block (Salmon et al., SC 2011) at counter {first + t, 0, 0, 0} with key
 * {seed, stream}; with outputs w0, w1:
 *   region_a != region_b: a = floor(w0 * |A| / 2^64), b = floor(w1 * |B| / 2^64)
 *   region_a == region_b: a = floor(w0 * |A| / 2^64), b' = floor(w1 * (|A|-1) / 2^64),
 *                         b = b' + (b' >= a), then ordered so that a < b.
 * pa[t], pb[t] receive the grid point ids of the region-local indices a, b.
 * pa/pb are device or host memory (out_is_device).
 */
cc_status cc_sample_pairs(cc_ctx* ctx, int32_t region_a, int32_t region_b, uint64_t seed,
                          uint64_t stream, uint64_t first, int64_t n_pairs, uint32_t* pa,
                          uint32_t* pb, int out_is_device);

/*
 * Quasi-random (low-discrepancy) point pairs between two box regions (Section
 * 3.1 names Halton and plastic-type low-discrepancy sequences as alternatives
 * to uniform random samples in the 6D space of a brick pair). Pair t takes the
 * point index j = first + t + 1 (first + n_pairs < 2^40) and a 6D point u:
 *   CC_LDS_HALTON  u_d = radical inverse of j in base (2, 3, 5, 7, 11, 13)[d]:
 *                  u_d = N_d / b^K with N_d the K base-b digits of j reversed;
 *                  c_d = floor(N_d * ext_d / b^K) in exact integer arithmetic.
 *   CC_LDS_R6      alpha_d = phi^-(d+1), phi the real root of x^7 = x + 1 (the
 *                  6D generalisation of the plastic number), as the nearest
 *                  doubles; u_d = frac(0.5 + j * alpha_d) and c_d = min(floor(
 *                  u_d * ext_d), ext_d - 1), each IEEE double operation rounded
 *                  once (no fused multiply-add).
 * ext_0..2 are the extents of region A's box and ext_3..5 of region B's; the
 * region-local indices are a = c_0 + ext_0 (c_1 + ext_1 c_2) and b likewise
 * from c_3..5. For region_a == region_b: if a == b then b = (b + 1) mod |A|,
 * then (a, b) is ordered so that a < b. pa[t], pb[t] receive the grid point
 * ids; device or host memory (out_is_device).
 */
#define CC_LDS_HALTON 1
#define CC_LDS_R6 2
cc_status cc_sample_pairs_lds(cc_ctx* ctx, int32_t region_a, int32_t region_b, int kind,
                              uint64_t first, int64_t n_pairs, uint32_t* pa, uint32_t* pb,
                              int out_is_device);

/* ------------------------------------------------------------------ evaluation */

/*
 * Evaluate one measure on a batch of point pairs (Section 3.2): out[t] =
 * measure(field_a point pa[t], field_b point pb[t]). The fields must have the
 * same member count. pa/pb are grid point ids (pairs_on_device says where
 * they live), out is float[n_pairs] (out_on_device). Pearson/Spearman use
 * fp32 (CC_FP32, CC_BF16, CC_FP8_E4M3) or the compensated Dot2 product
 * (CC_FP32_DOT2) of the fp32 planes. MI is in nats. An out-of-range
 * point id returns CC_ERR_INVALID_ARG (device-side check, reported by this
 * call when out is host memory, else by cc_sync).
 */
cc_status cc_eval_pairs(cc_ctx* ctx, int32_t field_a, int32_t field_b, const cc_params* params,
                        const uint32_t* pa, const uint32_t* pb, int64_t n_pairs,
                        int pairs_on_device, float* out, int out_on_device);

/*
 * KSG with its per-sample neighbour counts, for bit-exact verification
 * (Section 3.2). nx, ny are int32 [n_pairs][n] in the fields' member order
 * (n_x,i = 1 + #{j != i : |x_i - x_j| < eps_i}); eps is float [n_pairs][n]
 * (k-th smallest Chebyshev distance) or NULL. All outputs are host memory;
 * pa/pb are host memory.
 */
cc_status cc_ksg_counts(cc_ctx* ctx, int32_t field_a, int32_t field_b, int32_t k,
                        const uint32_t* pa, const uint32_t* pb, int64_t n_pairs, float* out,
                        int32_t* nx, int32_t* ny, float* eps);

/*
 * Per-region-pair extremes of a measure over candidate pair batches
 * (Section 3: max of point-to-point correlations per brick pair; Section 3.1:
 * batched evaluation across brick pairs). Segment s covers pairs
 * seg_offsets[s] .. seg_offsets[s+1]-1 of pa/pb (grid point ids of one field),
 * seg_offsets has n_seg + 1 host entries. out[s] (host) gets max/min and
 * argmax/argmin as batch indices t. values (float[n_pairs], device, or NULL)
 * receives every evaluated value.
 */
cc_status cc_segment_extremes(cc_ctx* ctx, int32_t field_id, const cc_params* params,
                              const uint32_t* pa, const uint32_t* pb, int pairs_on_device,
                              const int64_t* seg_offsets, int n_seg, float* values,
                              cc_rp_result* out);

/*
 * Two-variable form (Section 4.3): pa[t] indexes field_id and pb[t]
 * field_b_id (same ensemble size). cc_segment_extremes(ctx, f, ...) equals
 * cc_segment_extremes2(ctx, f, f, ...).
 */
cc_status cc_segment_extremes2(cc_ctx* ctx, int32_t field_id, int32_t field_b_id,
                               const cc_params* params, const uint32_t* pa, const uint32_t* pb,
                               int pairs_on_device, const int64_t* seg_offsets, int n_seg,
                               float* values, cc_rp_result* out);

/*
 * All pairs between two regions (Section 4.2: exhaustive focus refinement of
 * a brick pair; Section 3: maximum per brick pair). Pair (a, b) has linear
 * index a * |B| + b with a, b region-local indices. When region_a ==
 * region_b only a < b is reduced (each unordered pair once, no self pairs).
 *   values  device float matrix [|A|][ld] (ld >= |B|) receiving every value
 *           (for a self pair the full square, diagonal included), or NULL.
 *   out     host cc_rp_result of the reduced pairs.
 * Measures: CC_PEARSON and CC_SPEARMAN. params->precision CC_FP32 runs the
 * FP32 SIMT contraction; CC_BF16 / CC_FP8_E4M3 run cc_all_pairs_topk with
 * topk = 0 (values must then be NULL). The regions may belong to different
 * fields with the same n (inter-variable correlation, Section 4.3).
 */
cc_status cc_all_pairs(cc_ctx* ctx, int32_t region_a, int32_t region_b, const cc_params* params,
                       float* values, int64_t ld, cc_rp_result* out);

/*
 * Certificate of a reduced-precision all-pairs evaluation.
 *   bound          stated |approximate - refined| bound for every pair:
 *                  2e + e^2 + (1 + e)^2 2^-12 + 2^-20 with e the largest
 *                  per-point quantization error norm of the two regions
 *   threshold_max  pairs were re-evaluated when their approximate value could
 *                  reach this (= refined max - bound after the second pass)
 *   threshold_min  the same for the minimum (refined min + bound)
 *   certified_max  1 when every pair that could exceed out->max was re-evaluated,
 *                  so out->max is the exact maximum of the fp32 planes
 *   certified_min  likewise for out->min
 *   refined_pairs  pairs re-evaluated in compensated fp32 (Dot2)
 */
typedef struct {
    float bound;
    float threshold_max;
    float threshold_min;
    int32_t certified_max;
    int32_t certified_min;
    int64_t refined_pairs;
} cc_mixed_info;

/*
 * All pairs between two regions in reduced precision with exact extremes and
 * the top-`topk` list (project addition to Section 4.2's focus refinement).
 * params->precision CC_BF16 or CC_FP8_E4M3 (per-point scale 448/max|z|):
 * the contraction runs on the tensor cores with FP32 accumulation and yields
 * per-(row, 32-column chunk) approximate extremes; the top chunks and then
 * every chunk that could beat the best re-evaluated value within `bound` are
 * re-evaluated in compensated fp32 (Dot2, Ogita-Rump-Oishi 2005). out gets the
 * refined max/min (same index convention and self-pair rule as cc_all_pairs);
 * ids/vals (host, topk entries, may be NULL when topk == 0) the topk largest
 * refined values in descending order with their linear pair indices (missing
 * entries: value -inf, id UINT64_MAX). 0 <= topk <= 4096. info (host, may be
 * NULL) receives the certificate. Requires |A| * |B| < 2^32.
 * cc_all_pairs with precision CC_BF16 / CC_FP8_E4M3 is this call with topk = 0.
 */
cc_status cc_all_pairs_topk(cc_ctx* ctx, int32_t region_a, int32_t region_b,
                            const cc_params* params, int topk, uint64_t* ids, float* vals,
                            cc_rp_result* out, cc_mixed_info* info);

/*
 * The approximate values behind cc_all_pairs_topk, for stating their error
 * (project addition to Section 4.2's focus refinement). Runs the same
 * quantization and tensor-core contraction as cc_all_pairs_topk with the same
 * params and returns, per row a of region A and per chunk c of 32 consecutive
 * columns b = 32c .. 32c + 31 of region B, the largest and smallest
 * approximate value r~(a, b) of the chunk: cmax, cmin are host float
 * [ceil(|B| / 32)][|A|] (chunk-major). For a self region pair only b > a is
 * included; a chunk with no included pair holds -inf (cmax) and +inf (cmin).
 * *bound (host) receives the bound B that cc_all_pairs_topk certifies with:
 * |r~(a, b) - r(a, b)| <= B for every pair, r the value of the fp32 planes,
 * hence |cmax - max_b r| <= B and |cmin - min_b r| <= B per chunk.
 */
cc_status cc_all_pairs_approx(cc_ctx* ctx, int32_t region_a, int32_t region_b,
                              const cc_params* params, float* cmax, float* cmin, float* bound);

/* ------------------------------------------------- Bayesian optimal sampling (BOS) */

/*
 * Batched Bayesian optimal sampling of the brick-pair maxima (Section 3.1;
 * UCB kappa from Section 6). For every region pair a Gaussian process with
 * Matern nu = 5/2 covariance (ARD length scales 0.25 x the regions' extents
 * in voxels) models the objective measure over the 6D position space; each
 * round proposes `per_round` samples by UCB with kriging-believer batch
 * selection from the top `shortlist` entries of a fixed seeded pool of
 * `pool` continuous positions, maps them to voxels by probabilistic
 * reparameterization (floor + Bernoulli(fraction)), evaluates Pearson,
 * Spearman, binned MI and KSG at every sample in one persistent launch, and
 * conditions each GP on its new values. Signal variance, noise (1e-4 of it)
 * and the constant prior mean come from the first round's values unless a
 * prior mean per pool entry is set. The first `per_round` pool entries are
 * the initial random samples. Random numbers: Philox4x64-10 with key
 * {seed, 0xB05B05} for pool entry c of pair r at counters {c, r, 0, 0} and
 * {c, r, 1, 0} (position_d = u24(word_d) * (extent_d - 1), u24 = top 24 bits
 * / 2^24, fp32), and key {seed, 0xB0517D} for proposal j of round t at
 * {j, r, 2 + t, 0} and {j, r, 2 + t, 1}. In a self pair whose two voxels
 * coincide, the second moves to the next point of the region in enumeration
 * order (wrapping).
 */
typedef struct cc_bos cc_bos;

typedef struct {
    int32_t pool;       /* pool entries per region pair: power of two in [256, 8192] */
    int32_t per_round;  /* proposals per round and region pair, 1..32 */
    int32_t rounds;     /* rounds provisioned; per_round * rounds + shortlist <= pool */
    int32_t shortlist;  /* UCB shortlist for the batch selection, multiple of 16 in [16, 128] */
    float kappa;        /* UCB weight: mu + kappa * sigma */
    int32_t objective;  /* measure the GP models: CC_PEARSON .. CC_MI_KSG */
    int32_t k;          /* KSG neighbours (-1: ceil(3n/100)) */
    int32_t bins;       /* histogram bins, 2..16 */
    uint64_t seed;
    int32_t local_picks; /* local proposals per round from the second, 0 <= local_picks < per_round */
    float local_scale;   /* their spread per axis as a fraction of the region extent, (0, 1] */
} cc_bos_params;

/*
 * Local proposals (a project reading of how the acquisition is searched; the
 * paper names a global optimiser): with local_picks = L > 0, from the second
 * round on the first L proposals of a round are not taken from the pool but
 * perturb the two best samples so far (largest objective value, the earlier
 * sample on ties; proposal j uses incumbent j mod 2): theta_d = clip(theta_inc,d
 * + local_scale * extent_d * z_d, 0, extent_d - 1), z six standard normals by
 * Box-Muller from Philox blocks {j, r, 2 + t, 2} and {j, r, 2 + t, 3} (key
 * {seed, 0xB0517D}): for i = 0..2, u1 = (top 24 bits of word 2i + 1) / 2^24,
 * u2 = top 24 bits of word 2i+1 / 2^24, z_2i = sqrt(-2 ln u1) cos(2 pi u2),
 * z_2i+1 = ... sin. They are rounded, evaluated and reduced like every
 * proposal, but the GP is conditioned on the round's R - L pool proposals only
 * (all R in the first round). L = 0 is the plain reading.
 *
 * Create the sampling state for n_rp region pairs (rp_a[i], rp_b[i]) of one
 * field (host arrays). Device memory: pool * (6 + 2 + S) * 4 bytes per region
 * pair with S = per_round + (rounds - 1) (per_round - local_picks) GP
 * observations, plus per_round * rounds * 28 bytes of sample history.
 */
cc_status cc_bos_create(cc_ctx* ctx, int32_t field_id, const int32_t* rp_a, const int32_t* rp_b,
                        int n_rp, const cc_bos_params* params, cc_bos** out);

/*
 * Two-variable form (Section 4.3: sampling runs as for one field, but each
 * point pair takes its first point from field_id and its second from
 * field_b_id). Regions rp_a[i] belong to field_id, rp_b[i] to field_b_id; the
 * two fields need the same grid and ensemble size. Because the measure is no
 * longer symmetric in the two regions, the search of (A, B) and of (B, A)
 * are different entries of the inter-variable matrix, and no region pair is
 * a self pair (a voxel may pair with itself: its two variables differ).
 * cc_bos_create(ctx, f, ...) equals cc_bos_create2(ctx, f, f, ...).
 */
cc_status cc_bos_create2(cc_ctx* ctx, int32_t field_id, int32_t field_b_id, const int32_t* rp_a,
                         const int32_t* rp_b, int n_rp, const cc_bos_params* params,
                         cc_bos** out);

/*
 * Prior mean per pool entry, float [n_rp][pool] (e.g. a surrogate's
 * prediction); before the first round only. NULL restores the constant mean.
 */
cc_status cc_bos_set_prior(cc_ctx* ctx, cc_bos* bos, const float* prior, int prior_is_device);

/*
 * Run `rounds` rounds. use_graph != 0 captures one round into a CUDA graph on
 * first use and replays it. The evaluation kernel's launch shape is chosen by
 * timing a few shapes on the first call (cached per device and problem shape;
 * also in the file named by the environment variable CCORR_AUTOTUNE_CACHE).
 * Asynchronous.
 */
cc_status cc_bos_run(cc_ctx* ctx, cc_bos* bos, int rounds, int use_graph);

/*
 * Running extremes of the evaluated samples, host cc_rp_result [4][n_rp]
 * (measure-major: Pearson, Spearman, binned MI, KSG); argmax / argmin hold
 * (point_a << 32) | point_b, count the samples evaluated.
 */
cc_status cc_bos_results(cc_ctx* ctx, cc_bos* bos, cc_rp_result* out);

/*
 * Inspect region pair rp (host outputs, each may be NULL): pool [pool][6],
 * posterior mean and variance [pool], the GP's observed pool entries and
 * objective values [n_obs], the last round's point pairs [per_round] and
 * measure values [4][per_round]; *n_obs = GP observations so far.
 */
cc_status cc_bos_inspect(cc_ctx* ctx, cc_bos* bos, int rp, float* pool, float* mu, float* var,
                         int32_t* obs, float* y, uint32_t* pa, uint32_t* pb, float* vals,
                         int32_t* n_obs);

/*
 * Every sample evaluated so far for region pair rp, in order (round-major,
 * proposal j within a round): theta (host float [n][6], the continuous
 * position that was rounded, or NULL) and the objective measure's value
 * (host float [n], or NULL); *n_samples = rounds run x per_round.
 */
cc_status cc_bos_samples(cc_ctx* ctx, cc_bos* bos, int rp, float* theta, float* y,
                         int32_t* n_samples);

/* Release the sampling state. */
cc_status cc_bos_destroy(cc_ctx* ctx, cc_bos* bos);

/* ------------------------------------------------------------- learned surrogate */

/*
 * A small pairwise network that predicts a measure (e.g. KSG MI) from two
 * points' member vectors, the network the paper's Section 7 proposes as
 * future work. Used as the BOS prior mean (cc_bos_set_prior) and to screen all
 * pairs of a region pair; every reported maximum comes from exact evaluation.
 *   encoder  z (n) -> h1 = GELU(W1 z + b1) (128) -> e = W2 h1 + b2 (64)
 *   head     x = [e_i, e_j, |e_i - e_j|, off] (195) -> h3 = GELU(W3 x + b3)
 *            (128) -> y = w4 . h3 + b4, prediction = y * sd + mean
 * z = (v - mean) / sample std of the point's members; off = (position_j -
 * position_i) / (X, Y, Z); GELU = 0.5 x (1 + erf(x / sqrt 2)). Parameters are
 * one flat fp32 vector: W1 (128 x n, row-major), b1, W2 (64 x 128), b2,
 * W3 (128 x 195), b3, w4 (128), b4 -- 46,401 values for n = 100. Training:
 * MSE on targets standardized by their mean and sd, Adam (beta 0.9 / 0.999,
 * eps 1e-8) on fp32 master weights, BF16 weights and activations in every
 * contraction with fp32 accumulation, each pair's order swapped with
 * probability 1/2.
 */
typedef struct cc_sur cc_sur;

/* New surrogate for n-member fields with seeded N(0, 1/fan_in) weights. */
cc_status cc_sur_create(cc_ctx* ctx, int n_members, uint64_t seed, cc_sur** out);

/* Replace the parameters (host, flat layout above); resets the Adam state. */
cc_status cc_sur_set_params(cc_ctx* ctx, cc_sur* sur, const float* params);

/* Copy the parameters out (params may be NULL) and report count and target scale. */
cc_status cc_sur_get_params(cc_ctx* ctx, cc_sur* sur, float* params, int64_t* n_params,
                            float* target_mean, float* target_sd);

/* Set the target standardization (mean, sd > 0) used by the loss and predictions. */
cc_status cc_sur_set_target_scale(cc_ctx* ctx, cc_sur* sur, float mean, float sd);

/*
 * Loss (mean squared error on standardized targets) and its gradient (host,
 * flat layout) for one batch of pairs of field_id, without swapping or
 * updating. pa, pb, target, grad are host arrays.
 */
cc_status cc_sur_loss_grad(cc_ctx* ctx, cc_sur* sur, int32_t field_id, const uint32_t* pa,
                           const uint32_t* pb, const float* target, int64_t n_pairs, float* loss,
                           float* grad);

/*
 * Train for `epochs` epochs on pairs (pa[t], pb[t]) of field_id with target
 * values target[t] (host or device, on_device); the target mean and sd of
 * this set become the standardization. Mini-batches of `batch` pairs in a
 * seeded random order per epoch, learning rate lr. epoch_loss (host, epochs
 * entries, may be NULL) receives the mean standardized training loss.
 */
cc_status cc_sur_train(cc_ctx* ctx, cc_sur* sur, int32_t field_id, const uint32_t* pa,
                       const uint32_t* pb, const float* target, int64_t n_pairs, int on_device,
                       int epochs, int batch, float lr, uint64_t seed, float* epoch_loss);

/* Predictions for a batch of point pairs of field_id (host or device arrays). */
cc_status cc_sur_predict(cc_ctx* ctx, cc_sur* sur, int32_t field_id, const uint32_t* pa,
                         const uint32_t* pb, int64_t n_pairs, int pairs_on_device, float* out,
                         int out_on_device);

/*
 * Screen all pairs of two regions of one field: the topk (1..8192) largest
 * predictions in descending order, with linear pair indices a * |B| + b (host
 * arrays). Self region pairs consider a < b only. The head's first layer is
 * split so each point's projections are computed once.
 */
cc_status cc_sur_screen(cc_ctx* ctx, cc_sur* sur, int32_t region_a, int32_t region_b, int topk,
                        uint64_t* ids, float* preds);

/*
 * Surrogate-screened region-pair extremes: screen all pairs of two regions
 * (as cc_sur_screen), keep the `budget` pairs with the largest predictions
 * (ties at the cut may add a few; budget in [1, 2^24]), evaluate exactly those
 * pairs with `params` (any measure, as cc_eval_pairs) and return their exact
 * max / argmax / min / argmin in *out; argmax and argmin are linear pair
 * indices a * |B| + b, count is the number of pairs evaluated exactly. The
 * surrogate only chooses which pairs are evaluated: every reported value is
 * an exact evaluation. The maximum over the whole region pair is found
 * whenever its pair ranks within the budget in the surrogate's ordering.
 */
cc_status cc_sur_screen_verify(cc_ctx* ctx, cc_sur* sur, int32_t region_a, int32_t region_b,
                               int64_t budget, const cc_params* params, cc_rp_result* out);

/* Release the surrogate. */
cc_status cc_sur_destroy(cc_ctx* ctx, cc_sur* sur);

/* ------------------------------------------------------------ allocation-free form */

/*
 * All-pairs extremes without any device allocation. The paper has no
 * counterpart: this exists for callers that must not allocate device memory
 * while they run -- e.g. an interactive viewer's per-frame loop, or a host
 * application that owns all device memory in its own pool -- because
 * cudaMalloc may synchronise the whole device and fragments such pools.
 *
 * Same arithmetic as cc_all_pairs with measure CC_PEARSON/CC_SPEARMAN and
 * CC_FP32, but the caller supplies the standardized planes, so no context or
 * loaded field is needed:
 *   za, zb  device, member-major fp32 planes [nk][lda] / [nk][ldb]: column a
 *           holds the unit-norm centred member vector of point a (for
 *           Spearman: of its average ranks), rows n..nk-1 zero. 16-byte
 *           aligned; lda >= 128 * ceil(na / 128) and ldb >= 128 * ceil(nb /
 *           128), both multiples of 4, padding columns readable.
 *   nk      member count rounded up to a multiple of 8.
 *   na, nb  points per plane. self != 0 reduces only pairs a < b and needs
 *           za == zb, na == nb, lda == ldb.
 *   values  optional device matrix [na][ldv] (ldv >= nb) of every value.
 *   out     DEVICE pointer to one cc_rp_result (linear index a * nb + b).
 *   stream  cudaStream_t to run on (NULL: the default stream). Asynchronous.
 * Scratch is a file-scope device array of 65,536 tile partials (2.5 MiB,
 * held by every GPU that loads the library until the process exits), so at
 * most 65,536 tiles of 128 x 128 pairs: ceil(na/128) * ceil(nb/128) beyond
 * that returns CC_ERR_INVALID_ARG before any work is queued. The first call
 * on a device resolves the array's device address with that device current
 * (once per device); make that first call before any stream capture. Every
 * call shares the array: each call overwrites all partials it reads, so
 * nothing needs clearing, but calls whose work overlaps on the GPU race and
 * must be ordered (same stream, or events). Calls no cudaMalloc or cudaFree.
 * Returns CC_ERR_INVALID_ARG for bad sizes or alignment, CC_ERR_CUDA if a
 * launch fails.
 */
cc_status cc_all_pairs_static(const float* za, int64_t lda, const float* zb, int64_t ldb, int nk,
                              int64_t na, int64_t nb, int self, float* values, int64_t ldv,
                              cc_rp_result* out, void* stream);

/* ------------------------------------------------------------------ instrumentation */

/*
 * Number of kernels this library has launched in the process so far (all
 * contexts). Lets a caller count the library's launches inside a timed
 * region. Not part of the method.
 */
cc_status cc_launch_count(uint64_t* count);

#ifdef __cplusplus
}
#endif
#endif /* CCORR_H */
