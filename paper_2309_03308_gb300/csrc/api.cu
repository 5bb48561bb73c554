// C ABI of the ccorr library (declared in include/ccorr.h): context, field
// ingest, regions, pair sampling and measure evaluation. Host code only; the
// arithmetic runs in the kernels of prep.cu, pairs.cu and allpairs.cu.
#include <math.h>
#include <stdarg.h>
#include <stdio.h>
#include <string.h>

#include <algorithm>
#include <atomic>
#include <vector>

#include "internal.cuh"

using namespace cc;

namespace cc {

static std::atomic<uint64_t> g_launches{0};
void note_launch(int kernels) { g_launches.fetch_add((uint64_t)kernels); }

int sm_count() {
    int dev = 0, sms = 0;
    if (cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess ||
        sms < 1)
        sms = 1;
    return sms;
}

// psi(m) for integer m >= 1 (Eq. 2): psi(1) = -gamma, psi(m+1) = psi(m) + 1/m.
double digamma_int_host(int m) {
    long double s = -0.577215664901532860606512090082402431L;
    for (int j = 1; j < m; ++j) s += 1.0L / (long double)j;
    return (double)s;
}

}  // namespace cc

namespace {

cc_status fail(cc_ctx* c, cc_status s, const char* fmt, ...) __attribute__((format(printf, 3, 4)));
cc_status fail(cc_ctx* c, cc_status s, const char* fmt, ...) {
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

cc_status cuda_fail(cc_ctx* c, cudaError_t e, const char* where) {
    cudaGetLastError();
    return fail(c, e == cudaErrorMemoryAllocation ? CC_ERR_OOM : CC_ERR_CUDA, "%s: %s", where,
                cudaGetErrorString(e));
}

#define CK(call)                                                  \
    do {                                                          \
        cudaError_t _e = (call);                                  \
        if (_e != cudaSuccess) return cuda_fail(ctx, _e, #call);  \
    } while (0)

int round_up(int v, int m) { return (v + m - 1) / m * m; }

Field* get_field(cc_ctx* ctx, int32_t id) {
    if (id < 0 || id >= (int32_t)ctx->fields.size()) return nullptr;
    return ctx->fields[id].get();
}
Region* get_region(cc_ctx* ctx, int32_t id) {
    if (id < 0 || id >= (int32_t)ctx->regions.size()) return nullptr;
    Region* r = ctx->regions[id].get();
    if (!r || !get_field(ctx, r->field)) return nullptr;
    return r;
}

// Device status word: read, reset, map to cc_status.
// the library status of a device status word already read back (clears the
// device word when it holds an error)
cc_status status_value(cc_ctx* ctx, int s) {
    if (s == DEV_OK) return CC_OK;
    CK(cudaMemsetAsync(ctx->status.p, 0, sizeof(int), ctx->stream));
    switch (s) {
        case DEV_BAD_INDEX: return fail(ctx, CC_ERR_INVALID_ARG, "point id out of range");
        case DEV_NONFINITE: return fail(ctx, CC_ERR_NONFINITE, "field holds NaN or Inf");
        case DEV_TIMEOUT: return fail(ctx, CC_ERR_TIMEOUT, "device-side wait timed out");
    }
    return fail(ctx, CC_ERR_CUDA, "device status %d", s);
}

cc_status take_status(cc_ctx* ctx) {
    int s = 0;
    CK(cudaMemcpyAsync(&s, ctx->status.p, sizeof(int), cudaMemcpyDeviceToHost, ctx->stream));
    CK(cudaStreamSynchronize(ctx->stream));
    return status_value(ctx, s);
}

// fixed-point tables (2^40 scale) of psi(m) and m ln m for m = 0..n
cc_status table(cc_ctx* ctx, std::map<int, std::unique_ptr<DevMem>>& cache, int n, bool psi,
                const int64_t** out) {
    auto it = cache.find(n);
    if (it == cache.end()) {
        std::vector<long long> h(n + 1, 0);
        long double acc = -0.577215664901532860606512090082402431L;
        for (int m = 1; m <= n; ++m) {
            if (psi) {
                h[m] = llrintl(acc * (long double)kFixScale);
                acc += 1.0L / (long double)m;
            } else {
                h[m] = llrintl((long double)m * logl((long double)m) * (long double)kFixScale);
            }
        }
        auto buf = std::make_unique<DevMem>();
        CK(buf->alloc(sizeof(long long) * (n + 1)));
        CK(cudaMemcpyAsync(buf->p, h.data(), sizeof(long long) * (n + 1), cudaMemcpyHostToDevice,
                           ctx->stream));
        CK(cudaStreamSynchronize(ctx->stream));
        it = cache.emplace(n, std::move(buf)).first;
    }
    *out = it->second->as<int64_t>();
    return CC_OK;
}

cc_status ensure_bins(cc_ctx* ctx, Field& f, int B) {
    if (f.bins.count(B) && f.bins_version[B] == f.version) return CC_OK;
    const int64_t* clogc = nullptr;
    cc_status s = table(ctx, ctx->clogc_fix, f.n, false, &clogc);
    if (s) return s;
    if (!f.bins.count(B)) {
        auto b = std::make_unique<DevMem>();
        auto h = std::make_unique<DevMem>();
        CK(b->alloc((size_t)f.P * f.n_pad));
        CK(h->alloc(sizeof(int64_t) * f.P));
        f.bins[B] = std::move(b);
        f.hmarg[B] = std::move(h);
    }
    CK(launch_bins(f, B, clogc, f.bins[B]->as<uint8_t>(), f.hmarg[B]->as<int64_t>(), ctx->stream));
    f.bins_version[B] = f.version;
    return CC_OK;
}

// Stage a caller array on the device (no copy when it already is there).
template <class T>
cc_status stage(cc_ctx* ctx, DevMem& buf, const T* src, int64_t count, int on_device,
                const T** dev) {
    if (on_device) {
        *dev = src;
        return CC_OK;
    }
    CK(buf.ensure(sizeof(T) * (size_t)std::max<int64_t>(count, 1)));
    if (count > 0)
        CK(cudaMemcpyAsync(buf.p, src, sizeof(T) * count, cudaMemcpyHostToDevice, ctx->stream));
    *dev = buf.as<T>();
    return CC_OK;
}

cc_status check_params(cc_ctx* ctx, const cc_params* p, int n, int* k_out) {
    if (!p) return fail(ctx, CC_ERR_INVALID_ARG, "params is NULL");
    if (p->flags != 0) return fail(ctx, CC_ERR_INVALID_ARG, "params.flags must be 0");
    if (p->measure < CC_PEARSON || p->measure > CC_MI_KSG)
        return fail(ctx, CC_ERR_INVALID_ARG, "unknown measure %d", p->measure);
    if (p->precision < CC_FP32 || p->precision > CC_FP32_DOT2)
        return fail(ctx, CC_ERR_INVALID_ARG, "unknown precision %d", p->precision);
    if (p->measure == CC_MI_BINNED && (p->bins < 2 || p->bins > 16))
        return fail(ctx, CC_ERR_INVALID_ARG, "bins must be in [2, 16], got %d", p->bins);
    if (p->measure == CC_MI_KSG) {
        int k = p->k == -1 ? (3 * n + 99) / 100 : p->k;
        if (k < 1 || k > n - 1 || k > 32)
            return fail(ctx, CC_ERR_INVALID_ARG, "k must be in [1, min(n-1, 32)], got %d", k);
        if (k_out) *k_out = k;
    }
    return CC_OK;
}

// Evaluate a measure into a device buffer `out` (pairs already on device).
cc_status eval_device(cc_ctx* ctx, Field& fa, Field& fb, const cc_params* p, int k,
                      const uint32_t* pa, const uint32_t* pb, int64_t N, float* out) {
    int* st = ctx->status.as<int>();
    const bool dot2 = p->precision == CC_FP32_DOT2;
    switch (p->measure) {
        case CC_PEARSON:
        case CC_SPEARMAN: {
            const bool sp = p->measure == CC_SPEARMAN;
            const float* A = sp ? fa.rhat.as<float>() : fa.zhat.as<float>();
            const float* B = sp ? fb.rhat.as<float>() : fb.zhat.as<float>();
            if (dot2)
                CK(launch_dot2_pairs(A, fa.P, B, fb.P, fa.n_pad, fa.n, pa, pb, N, out, st,
                                     ctx->stream));
            else
                CK(launch_pearson_pairs(A, fa.P, B, fb.P, fa.n_pad, pa, pb, N, out, st,
                                        ctx->stream));
            break;
        }
        case CC_MI_BINNED: {
            cc_status s = ensure_bins(ctx, fa, p->bins);
            if (!s && &fb != &fa) s = ensure_bins(ctx, fb, p->bins);
            if (s) return s;
            const int64_t* clogc = nullptr;
            s = table(ctx, ctx->clogc_fix, fa.n, false, &clogc);
            if (s) return s;
            CK(launch_hist_pairs(fa.bins[p->bins]->as<uint8_t>(), fa.hmarg[p->bins]->as<int64_t>(),
                                 fa.P, fb.bins[p->bins]->as<uint8_t>(),
                                 fb.hmarg[p->bins]->as<int64_t>(), fb.P, fa.n, fa.n_pad, p->bins,
                                 clogc, pa, pb, N, out, st, ctx->stream));
            break;
        }
        case CC_MI_KSG: {
            const int64_t* psi = nullptr;
            cc_status s = table(ctx, ctx->psi_fix, fa.n, true, &psi);
            if (s) return s;
            CK(launch_ksg_pairs(fa, fb, k, psi, pa, pb, N, out, nullptr, nullptr, nullptr, st,
                                ctx->stream));
            break;
        }
    }
    return CC_OK;
}

cc_status ensure_region_planes(cc_ctx* ctx, Region& r) {
    Field& f = *ctx->fields[r.field];
    if (r.zT.p && r.planes_version == f.version) return CC_OK;
    if (!r.zT.p) {
        r.nk = round_up(f.n, 8);
        r.np_pad = (r.np + 127) / 128 * 128;
        CK(r.zT.alloc(sizeof(float) * (size_t)r.nk * r.np_pad));
        CK(r.rT.alloc(sizeof(float) * (size_t)r.nk * r.np_pad));
    }
    CK(launch_region_planes(f, r, ctx->stream));
    r.planes_version = f.version;
    return CC_OK;
}

cc_status make_region(cc_ctx* ctx, int32_t field_id, const cc_box& b, int32_t* id) {
    Field* f = get_field(ctx, field_id);
    if (!f) return fail(ctx, CC_ERR_INVALID_ARG, "unknown field %d", field_id);
    if (b.x0 < 0 || b.y0 < 0 || b.z0 < 0 || b.x1 > f->X || b.y1 > f->Y || b.z1 > f->Z ||
        b.x0 >= b.x1 || b.y0 >= b.y1 || b.z0 >= b.z1)
        return fail(ctx, CC_ERR_INVALID_ARG, "box (%d,%d,%d)-(%d,%d,%d) outside field or empty",
                    b.x0, b.y0, b.z0, b.x1, b.y1, b.z1);
    auto r = std::make_unique<Region>();
    r->field = field_id;
    r->box = b;
    r->np = (int64_t)(b.x1 - b.x0) * (b.y1 - b.y0) * (b.z1 - b.z0);
    r->pts_host.reserve(r->np);
    for (int z = b.z0; z < b.z1; ++z)
        for (int y = b.y0; y < b.y1; ++y)
            for (int x = b.x0; x < b.x1; ++x)
                r->pts_host.push_back((uint32_t)(x + (int64_t)f->X * (y + (int64_t)f->Y * z)));
    CK(r->pts.alloc(sizeof(uint32_t) * r->np));
    CK(cudaMemcpyAsync(r->pts.p, r->pts_host.data(), sizeof(uint32_t) * r->np,
                       cudaMemcpyHostToDevice, ctx->stream));
    CK(cudaStreamSynchronize(ctx->stream));
    *id = (int32_t)ctx->regions.size();
    ctx->regions.push_back(std::move(r));
    return CC_OK;
}

}  // namespace

extern "C" {

cc_status cc_create(int device, void* stream, cc_ctx** out) {
    if (!out) return CC_ERR_INVALID_ARG;
    *out = nullptr;
    int count = 0;
    if (cudaGetDeviceCount(&count) != cudaSuccess || device < 0 || device >= count) {
        cudaGetLastError();
        return CC_ERR_INVALID_ARG;
    }
    cc_ctx* ctx = new (std::nothrow) cc_ctx();
    if (!ctx) return CC_ERR_OOM;
    ctx->device = device;
    cudaError_t e = cudaSetDevice(device);
    if (e == cudaSuccess && stream) {
        ctx->stream = (cudaStream_t)stream;
    } else if (e == cudaSuccess) {
        e = cudaStreamCreateWithFlags(&ctx->stream, cudaStreamNonBlocking);
        ctx->own_stream = e == cudaSuccess;
    }
    if (e == cudaSuccess) e = ctx->status.alloc(sizeof(int) * 4);
    if (e == cudaSuccess) e = cudaMemsetAsync(ctx->status.p, 0, sizeof(int) * 4, ctx->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(ctx->stream);
    if (e != cudaSuccess) {
        cudaGetLastError();
        if (ctx->own_stream) cudaStreamDestroy(ctx->stream);
        delete ctx;
        return e == cudaErrorMemoryAllocation ? CC_ERR_OOM : CC_ERR_CUDA;
    }
    *out = ctx;
    return CC_OK;
}

cc_status cc_destroy(cc_ctx* ctx) {
    if (!ctx) return CC_ERR_INVALID_ARG;
    cudaSetDevice(ctx->device);
    cudaStreamSynchronize(ctx->stream);
    cudaStream_t st = ctx->stream;
    bool own = ctx->own_stream;
    delete ctx;
    if (own) cudaStreamDestroy(st);
    return CC_OK;
}

const char* cc_last_error(const cc_ctx* ctx) { return ctx ? ctx->err.c_str() : "null context"; }

cc_status cc_sync(cc_ctx* ctx) {
    if (!ctx) return CC_ERR_INVALID_ARG;
    CK(cudaStreamSynchronize(ctx->stream));
    return take_status(ctx);
}

cc_status cc_load_field(cc_ctx* ctx, const float* data, int data_is_device, int X, int Y, int Z,
                        int n, int32_t* field_id) {
    if (!ctx) return CC_ERR_INVALID_ARG;
    if (!data || !field_id) return fail(ctx, CC_ERR_INVALID_ARG, "NULL data or field_id");
    if (X < 1 || Y < 1 || Z < 1 || n < 2 || n > 1024)
        return fail(ctx, CC_ERR_INVALID_ARG, "need X,Y,Z >= 1 and 2 <= n <= 1024");
    const int64_t P = (int64_t)X * Y * Z;
    if (P > 0xFFFFFFFFll) return fail(ctx, CC_ERR_INVALID_ARG, "more than 2^32 grid points");
    CK(cudaSetDevice(ctx->device));
    auto f = std::make_unique<Field>();
    f->X = X;
    f->Y = Y;
    f->Z = Z;
    f->n = n;
    f->n_pad = 32;
    while (f->n_pad < n) f->n_pad *= 2;  // power of two: the per-point sort is bitonic
    f->P = P;
    const size_t cells = (size_t)P * f->n_pad;
    CK(f->vals.alloc(cells * 4));
    CK(f->sorted.alloc(cells * 4));
    CK(f->perm.alloc(cells * 2));
    CK(f->rank2.alloc(cells * 2));
    CK(f->zhat.alloc(cells * 4));
    CK(f->rhat.alloc(cells * 4));
    CK(f->mean.alloc(8 * P));
    CK(f->ss.alloc(8 * P));
    const float* src = data;
    DevMem staging;
    if (!data_is_device) {
        CK(staging.alloc(sizeof(float) * (size_t)P * n));
        CK(cudaMemcpyAsync(staging.p, data, sizeof(float) * (size_t)P * n, cudaMemcpyHostToDevice,
                           ctx->stream));
        src = staging.as<float>();
    }
    CK(launch_ingest(src, n, P, P, f->n_pad, f->vals.as<float>(), ctx->status.as<int>(),
                     ctx->stream));
    cc_status s = take_status(ctx);  // synchronises: staging may be released after this
    if (s) return s;
    CK(launch_point_prep(*f, ctx->stream));
    *field_id = (int32_t)ctx->fields.size();
    ctx->fields.push_back(std::move(f));
    return CC_OK;
}

cc_status cc_aggregate_field(cc_ctx* ctx, int32_t field_id, int bx, int by, int bz, int mode,
                             int32_t* out_field_id) {
    if (!ctx) return CC_ERR_INVALID_ARG;
    Field* f = get_field(ctx, field_id);
    if (!f || !out_field_id || bx < 1 || by < 1 || bz < 1 ||
        (mode != CC_AGG_MEAN && mode != CC_AGG_MAX))
        return fail(ctx, CC_ERR_INVALID_ARG, "bad arguments");
    CK(cudaSetDevice(ctx->device));
    const int Xc = (f->X + bx - 1) / bx, Yc = (f->Y + by - 1) / by, Zc = (f->Z + bz - 1) / bz;
    const int64_t Pc = (int64_t)Xc * Yc * Zc;
    DevMem agg;
    CK(agg.alloc(sizeof(float) * (size_t)Pc * f->n));
    CK(launch_aggregate(*f, bx, by, bz, Xc, Yc, Pc, mode, agg.as<float>(), ctx->stream));
    const int n = f->n;  // f may move when the field list grows
    return cc_load_field(ctx, agg.as<float>(), 1, Xc, Yc, Zc, n, out_field_id);
}

constexpr int kUpdateChunks = 8;  // point ranges of a host-data update

cc_status cc_update_field(cc_ctx* ctx, int32_t field_id, const float* data, int data_is_device) {
    if (!ctx) return CC_ERR_INVALID_ARG;
    Field* f = get_field(ctx, field_id);
    if (!f || !data) return fail(ctx, CC_ERR_INVALID_ARG, "unknown field or NULL data");
    CK(cudaSetDevice(ctx->device));
    // bin planes already in use are rebuilt in the same pass (two bin counts)
    PrepBins pb;
    for (auto& kv : f->bins) {
        if (pb.count == 2) break;
        const int64_t* clogc = nullptr;
        cc_status s = table(ctx, ctx->clogc_fix, f->n, false, &clogc);
        if (s) return s;
        pb.clogc = (const long long*)clogc;
        pb.B[pb.count] = kv.first;
        pb.bins[pb.count] = kv.second->as<uint8_t>();
        pb.hmarg[pb.count] = f->hmarg[kv.first]->as<long long>();
        ++pb.count;
    }
    if (data_is_device) {
        CK(launch_ingest(data, f->n, f->P, f->P, f->n_pad, f->vals.as<float>(),
                         ctx->status.as<int>(), ctx->stream));
        CK(launch_point_prep(*f, ctx->stream, pb));
    } else {
        // Host data: the copy is cut into point ranges (one 2D copy of n
        // member rows each) on a second stream, and each range's ingest and
        // per-point pass start as soon as its copy has landed, so the
        // transfer overlaps the computation. The staging buffer keeps the
        // caller's member-major layout.
        const size_t bytes = sizeof(float) * (size_t)f->P * f->n;
        CK(f->staging.ensure(bytes));
        const int chunks = bytes >= ((size_t)64 << 20) ? kUpdateChunks : 1;
        if (!ctx->copy_stream)
            CK(cudaStreamCreateWithFlags(&ctx->copy_stream, cudaStreamNonBlocking));
        while ((int)ctx->copy_events.size() < kUpdateChunks + 1) {
            cudaEvent_t e;
            CK(cudaEventCreateWithFlags(&e, cudaEventDisableTiming));
            ctx->copy_events.push_back(e);
        }
        // the staging buffer may still be read by work queued before this call
        CK(cudaEventRecord(ctx->copy_events[kUpdateChunks], ctx->stream));
        CK(cudaStreamWaitEvent(ctx->copy_stream, ctx->copy_events[kUpdateChunks], 0));
        const int64_t step = (f->P + chunks - 1) / chunks;
        float* stg = f->staging.as<float>();
        for (int c = 0; c < chunks; ++c) {
            const int64_t p0 = c * step, pc = std::min<int64_t>(step, f->P - p0);
            if (pc <= 0) break;
            CK(cudaMemcpy2DAsync(stg + p0, sizeof(float) * (size_t)f->P, data + p0,
                                 sizeof(float) * (size_t)f->P, sizeof(float) * (size_t)pc,
                                 (size_t)f->n, cudaMemcpyHostToDevice, ctx->copy_stream));
            CK(cudaEventRecord(ctx->copy_events[c], ctx->copy_stream));
        }
        for (int c = 0; c < chunks; ++c) {
            const int64_t p0 = c * step, pc = std::min<int64_t>(step, f->P - p0);
            if (pc <= 0) break;
            CK(cudaStreamWaitEvent(ctx->stream, ctx->copy_events[c], 0));
            CK(launch_ingest(stg + p0, f->n, pc, f->P, f->n_pad,
                             f->vals.as<float>() + p0 * f->n_pad, ctx->status.as<int>(),
                             ctx->stream));
            CK(launch_point_prep(*f, ctx->stream, pb, p0, p0 + pc));
        }
    }
    f->version++;
    for (int i = 0; i < pb.count; ++i) f->bins_version[pb.B[i]] = f->version;
    return CC_OK;
}

cc_status cc_launch_count(uint64_t* count) {
    if (!count) return CC_ERR_INVALID_ARG;
    *count = g_launches.load();
    return CC_OK;
}

cc_status cc_free_field(cc_ctx* ctx, int32_t field_id) {
    if (!ctx) return CC_ERR_INVALID_ARG;
    if (!get_field(ctx, field_id)) return fail(ctx, CC_ERR_INVALID_ARG, "unknown field");
    CK(cudaStreamSynchronize(ctx->stream));
    ctx->fields[field_id].reset();
    for (auto& r : ctx->regions)
        if (r && r->field == field_id) r.reset();
    return CC_OK;
}

cc_status cc_get_plane(cc_ctx* ctx, int32_t field_id, int plane, int bins, const uint32_t* pts,
                       int64_t count, void* out) {
    if (!ctx) return CC_ERR_INVALID_ARG;
    Field* f = get_field(ctx, field_id);
    if (!f || !pts || !out || count < 0) return fail(ctx, CC_ERR_INVALID_ARG, "bad arguments");
    size_t esz;
    const unsigned char* base;
    switch (plane) {
        case CC_PLANE_RANK2: esz = 2; base = f->rank2.as<unsigned char>(); break;
        case CC_PLANE_SORTED: esz = 4; base = f->sorted.as<unsigned char>(); break;
        case CC_PLANE_ZHAT: esz = 4; base = f->zhat.as<unsigned char>(); break;
        case CC_PLANE_BINS: {
            if (bins < 2 || bins > 16) return fail(ctx, CC_ERR_INVALID_ARG, "bins in [2, 16]");
            cc_status s = ensure_bins(ctx, *f, bins);
            if (s) return s;
            esz = 1;
            base = f->bins[bins]->as<unsigned char>();
            break;
        }
        default: return fail(ctx, CC_ERR_INVALID_ARG, "unknown plane %d", plane);
    }
    std::vector<unsigned char> row((size_t)f->n * esz);
    for (int64_t i = 0; i < count; ++i) {
        if (pts[i] >= (uint64_t)f->P) return fail(ctx, CC_ERR_INVALID_ARG, "point id out of range");
        CK(cudaMemcpyAsync(row.data(), base + (size_t)pts[i] * f->n_pad * esz, row.size(),
                           cudaMemcpyDeviceToHost, ctx->stream));
        CK(cudaStreamSynchronize(ctx->stream));
        unsigned char* dst = (unsigned char*)out;
        if (plane == CC_PLANE_RANK2) {
            int32_t* d = (int32_t*)dst + i * f->n;
            const int16_t* s = (const int16_t*)row.data();
            for (int m = 0; m < f->n; ++m) d[m] = s[m];
        } else {
            memcpy(dst + (size_t)i * row.size(), row.data(), row.size());
        }
    }
    return CC_OK;
}

cc_status cc_define_regions(cc_ctx* ctx, int32_t field_id, const cc_box* boxes, int count,
                            int32_t* region_ids) {
    if (!ctx) return CC_ERR_INVALID_ARG;
    if (!boxes || !region_ids || count < 0) return fail(ctx, CC_ERR_INVALID_ARG, "bad arguments");
    for (int i = 0; i < count; ++i) {
        cc_status s = make_region(ctx, field_id, boxes[i], &region_ids[i]);
        if (s) return s;
    }
    return CC_OK;
}

cc_status cc_partition_regular(cc_ctx* ctx, int32_t field_id, int bx, int by, int bz,
                               int32_t* region_ids, int cap, int* count) {
    if (!ctx) return CC_ERR_INVALID_ARG;
    Field* f = get_field(ctx, field_id);
    if (!f || bx < 1 || by < 1 || bz < 1 || !count || (cap > 0 && !region_ids))
        return fail(ctx, CC_ERR_INVALID_ARG, "bad arguments");
    const int nx = (f->X + bx - 1) / bx, ny = (f->Y + by - 1) / by, nz = (f->Z + bz - 1) / bz;
    *count = nx * ny * nz;
    if (*count > cap) return fail(ctx, CC_ERR_INVALID_ARG, "cap %d < %d regions", cap, *count);
    int i = 0;
    for (int z = 0; z < f->Z; z += bz)
        for (int y = 0; y < f->Y; y += by)
            for (int x = 0; x < f->X; x += bx) {
                cc_box b{x, y, z, std::min(x + bx, f->X), std::min(y + by, f->Y),
                         std::min(z + bz, f->Z)};
                cc_status s = make_region(ctx, field_id, b, &region_ids[i++]);
                if (s) return s;
            }
    return CC_OK;
}

cc_status cc_region_info(cc_ctx* ctx, int32_t region_id, int64_t* npoints, cc_box* box) {
    if (!ctx) return CC_ERR_INVALID_ARG;
    Region* r = get_region(ctx, region_id);
    if (!r || !npoints) return fail(ctx, CC_ERR_INVALID_ARG, "unknown region %d", region_id);
    *npoints = r->np;
    if (box) *box = r->box;
    return CC_OK;
}

cc_status cc_sample_pairs(cc_ctx* ctx, int32_t region_a, int32_t region_b, uint64_t seed,
                          uint64_t stream, uint64_t first, int64_t n_pairs, uint32_t* pa,
                          uint32_t* pb, int out_is_device) {
    if (!ctx) return CC_ERR_INVALID_ARG;
    Region* ra = get_region(ctx, region_a);
    Region* rb = get_region(ctx, region_b);
    if (!ra || !rb || !pa || !pb || n_pairs < 0)
        return fail(ctx, CC_ERR_INVALID_ARG, "bad arguments");
    const int self = region_a == region_b;
    if (self && ra->np < 2) return fail(ctx, CC_ERR_INVALID_ARG, "self pair needs >= 2 points");
    uint32_t *da = pa, *db = pb;
    if (!out_is_device) {
        CK(ctx->pair_a.ensure(4 * (size_t)std::max<int64_t>(n_pairs, 1)));
        CK(ctx->pair_b.ensure(4 * (size_t)std::max<int64_t>(n_pairs, 1)));
        da = ctx->pair_a.as<uint32_t>();
        db = ctx->pair_b.as<uint32_t>();
    }
    CK(launch_sample_pairs(ra->pts.as<uint32_t>(), ra->np, rb->pts.as<uint32_t>(), rb->np, self,
                           seed, stream, first, n_pairs, da, db, ctx->stream));
    if (!out_is_device && n_pairs > 0) {
        CK(cudaMemcpyAsync(pa, da, 4 * n_pairs, cudaMemcpyDeviceToHost, ctx->stream));
        CK(cudaMemcpyAsync(pb, db, 4 * n_pairs, cudaMemcpyDeviceToHost, ctx->stream));
        CK(cudaStreamSynchronize(ctx->stream));
    }
    return CC_OK;
}

cc_status cc_sample_pairs_lds(cc_ctx* ctx, int32_t region_a, int32_t region_b, int kind,
                              uint64_t first, int64_t n_pairs, uint32_t* pa, uint32_t* pb,
                              int out_is_device) {
    if (!ctx) return CC_ERR_INVALID_ARG;
    Region* ra = get_region(ctx, region_a);
    Region* rb = get_region(ctx, region_b);
    if (!ra || !rb || !pa || !pb || n_pairs < 0 || (kind != CC_LDS_HALTON && kind != CC_LDS_R6))
        return fail(ctx, CC_ERR_INVALID_ARG, "bad arguments");
    if (first + (uint64_t)n_pairs >= (1ull << 40))
        return fail(ctx, CC_ERR_INVALID_ARG, "first + n_pairs must be below 2^40");
    const int self = region_a == region_b;
    if (self && ra->np < 2) return fail(ctx, CC_ERR_INVALID_ARG, "self pair needs >= 2 points");
    const cc_box& A = ra->box;
    const cc_box& B = rb->box;
    const int ext[6] = {A.x1 - A.x0, A.y1 - A.y0, A.z1 - A.z0,
                        B.x1 - B.x0, B.y1 - B.y0, B.z1 - B.z0};
    // alpha_d = phi^-(d+1), phi the real root of x^7 = x + 1: bisection in
    // extended precision, then rounded to double
    double alpha[6];
    {
        long double lo = 1.0L, hi = 2.0L;
        for (int i = 0; i < 200; ++i) {
            const long double mid = 0.5L * (lo + hi);
            const long double f = mid * mid * mid * mid * mid * mid * mid - mid - 1.0L;
            (f > 0.0L ? hi : lo) = mid;
        }
        const long double phi = 0.5L * (lo + hi);
        long double p = 1.0L;
        for (int d = 0; d < 6; ++d) {
            p /= phi;
            alpha[d] = (double)p;
        }
    }
    uint32_t *da = pa, *db = pb;
    if (!out_is_device) {
        CK(ctx->pair_a.ensure(4 * (size_t)std::max<int64_t>(n_pairs, 1)));
        CK(ctx->pair_b.ensure(4 * (size_t)std::max<int64_t>(n_pairs, 1)));
        da = ctx->pair_a.as<uint32_t>();
        db = ctx->pair_b.as<uint32_t>();
    }
    CK(launch_sample_lds(kind, ext, alpha, self, ra->pts.as<uint32_t>(), rb->pts.as<uint32_t>(),
                         first, n_pairs, da, db, ctx->stream));
    if (!out_is_device && n_pairs > 0) {
        CK(cudaMemcpyAsync(pa, da, 4 * n_pairs, cudaMemcpyDeviceToHost, ctx->stream));
        CK(cudaMemcpyAsync(pb, db, 4 * n_pairs, cudaMemcpyDeviceToHost, ctx->stream));
        CK(cudaStreamSynchronize(ctx->stream));
    }
    return CC_OK;
}

cc_status cc_eval_pairs(cc_ctx* ctx, int32_t field_a, int32_t field_b, const cc_params* params,
                        const uint32_t* pa, const uint32_t* pb, int64_t n_pairs,
                        int pairs_on_device, float* out, int out_on_device) {
    if (!ctx) return CC_ERR_INVALID_ARG;
    Field* fa = get_field(ctx, field_a);
    Field* fb = get_field(ctx, field_b);
    if (!fa || !fb) return fail(ctx, CC_ERR_INVALID_ARG, "unknown field");
    if (fa->n != fb->n) return fail(ctx, CC_ERR_INVALID_ARG, "fields differ in member count");
    if (!pa || !pb || !out || n_pairs < 0) return fail(ctx, CC_ERR_INVALID_ARG, "bad arguments");
    int k = 0;
    cc_status s = check_params(ctx, params, fa->n, &k);
    if (s) return s;
    if (n_pairs == 0) return CC_OK;
    CK(cudaSetDevice(ctx->device));
    const uint32_t *da, *db;
    if ((s = stage(ctx, ctx->pair_a, pa, n_pairs, pairs_on_device, &da))) return s;
    if ((s = stage(ctx, ctx->pair_b, pb, n_pairs, pairs_on_device, &db))) return s;
    float* dout = out;
    if (!out_on_device) {
        CK(ctx->vals_out.ensure(4 * (size_t)n_pairs));
        dout = ctx->vals_out.as<float>();
    }
    if ((s = eval_device(ctx, *fa, *fb, params, k, da, db, n_pairs, dout))) return s;
    if (!out_on_device) {
        CK(cudaMemcpyAsync(out, dout, 4 * n_pairs, cudaMemcpyDeviceToHost, ctx->stream));
        return take_status(ctx);
    }
    return CC_OK;
}

cc_status cc_ksg_counts(cc_ctx* ctx, int32_t field_a, int32_t field_b, int32_t k,
                        const uint32_t* pa, const uint32_t* pb, int64_t n_pairs, float* out,
                        int32_t* nx, int32_t* ny, float* eps) {
    if (!ctx) return CC_ERR_INVALID_ARG;
    Field* fa = get_field(ctx, field_a);
    Field* fb = get_field(ctx, field_b);
    if (!fa || !fb || fa->n != fb->n) return fail(ctx, CC_ERR_INVALID_ARG, "bad fields");
    if (!pa || !pb || !out || !nx || !ny || n_pairs < 0)
        return fail(ctx, CC_ERR_INVALID_ARG, "bad arguments");
    cc_params p{CC_MI_KSG, k, 0, 0, 0};
    int kk = 0;
    cc_status s = check_params(ctx, &p, fa->n, &kk);
    if (s) return s;
    if (n_pairs == 0) return CC_OK;
    const uint32_t *da, *db;
    if ((s = stage(ctx, ctx->pair_a, pa, n_pairs, 0, &da))) return s;
    if ((s = stage(ctx, ctx->pair_b, pb, n_pairs, 0, &db))) return s;
    const size_t cnt = (size_t)n_pairs * fa->n;
    CK(ctx->vals_out.ensure(4 * (size_t)n_pairs));
    CK(ctx->ksg_nx.ensure(4 * cnt));
    CK(ctx->ksg_ny.ensure(4 * cnt));
    CK(ctx->ksg_eps.ensure(4 * cnt));
    const int64_t* psi = nullptr;
    if ((s = table(ctx, ctx->psi_fix, fa->n, true, &psi))) return s;
    CK(launch_ksg_pairs(*fa, *fb, kk, psi, da, db, n_pairs, ctx->vals_out.as<float>(),
                        ctx->ksg_nx.as<int32_t>(), ctx->ksg_ny.as<int32_t>(),
                        ctx->ksg_eps.as<float>(), ctx->status.as<int>(), ctx->stream));
    CK(cudaMemcpyAsync(out, ctx->vals_out.p, 4 * n_pairs, cudaMemcpyDeviceToHost, ctx->stream));
    CK(cudaMemcpyAsync(nx, ctx->ksg_nx.p, 4 * cnt, cudaMemcpyDeviceToHost, ctx->stream));
    CK(cudaMemcpyAsync(ny, ctx->ksg_ny.p, 4 * cnt, cudaMemcpyDeviceToHost, ctx->stream));
    if (eps)
        CK(cudaMemcpyAsync(eps, ctx->ksg_eps.p, 4 * cnt, cudaMemcpyDeviceToHost, ctx->stream));
    return take_status(ctx);
}

cc_status cc_segment_extremes2(cc_ctx* ctx, int32_t field_id, int32_t field_b_id,
                               const cc_params* params, const uint32_t* pa, const uint32_t* pb,
                               int pairs_on_device, const int64_t* seg_offsets, int n_seg,
                               float* values, cc_rp_result* out) {
    if (!ctx) return CC_ERR_INVALID_ARG;
    Field* f = get_field(ctx, field_id);
    Field* g = get_field(ctx, field_b_id);
    if (!f || !g || !pa || !pb || !seg_offsets || !out || n_seg < 0)
        return fail(ctx, CC_ERR_INVALID_ARG, "bad arguments");
    if (f->n != g->n) return fail(ctx, CC_ERR_INVALID_ARG, "fields differ in member count");
    for (int s = 0; s < n_seg; ++s)
        if (seg_offsets[s + 1] < seg_offsets[s] || seg_offsets[0] != 0)
            return fail(ctx, CC_ERR_INVALID_ARG, "segment offsets must start at 0 and not decrease");
    const int64_t N = seg_offsets[n_seg];
    int k = 0;
    cc_status s = check_params(ctx, params, f->n, &k);
    if (s) return s;
    const uint32_t *da, *db;
    if ((s = stage(ctx, ctx->pair_a, pa, N, pairs_on_device, &da))) return s;
    if ((s = stage(ctx, ctx->pair_b, pb, N, pairs_on_device, &db))) return s;
    float* dv = values;
    if (!dv) {
        CK(ctx->vals_out.ensure(4 * (size_t)std::max<int64_t>(N, 1)));
        dv = ctx->vals_out.as<float>();
    }
    if ((s = eval_device(ctx, *f, *g, params, k, da, db, N, dv))) return s;
    // chunk table: [start, end) per chunk, first chunk per segment
    std::vector<int64_t> table_h;
    std::vector<int64_t> first_h(n_seg + 1);
    int64_t n_chunks = 0;
    for (int sg = 0; sg < n_seg; ++sg) {
        first_h[sg] = n_chunks;
        for (int64_t c = seg_offsets[sg]; c < seg_offsets[sg + 1]; c += kSegChunk) {
            table_h.push_back(c);
            table_h.push_back(std::min(c + kSegChunk, seg_offsets[sg + 1]));
            ++n_chunks;
        }
    }
    first_h[n_seg] = n_chunks;
    const size_t res_bytes = sizeof(Partial) * (std::max(n_seg, 1) + n_chunks);
    const size_t tab_bytes = sizeof(int64_t) * (table_h.size() + first_h.size());
    CK(ctx->rp_out.ensure(res_bytes + tab_bytes));
    Partial* dres = ctx->rp_out.as<Partial>();
    Partial* dpart = dres + std::max(n_seg, 1);
    int64_t* dtab = reinterpret_cast<int64_t*>(dpart + n_chunks);
    int64_t* dfirst = dtab + table_h.size();
    table_h.insert(table_h.end(), first_h.begin(), first_h.end());
    CK(cudaMemcpyAsync(dtab, table_h.data(), tab_bytes, cudaMemcpyHostToDevice, ctx->stream));
    CK(launch_segment_extremes(dv, dtab, n_chunks, dfirst, n_seg, dpart, dres, ctx->stream));
    std::vector<Partial> h(std::max(n_seg, 1));
    CK(cudaMemcpyAsync(h.data(), dres, sizeof(Partial) * n_seg, cudaMemcpyDeviceToHost,
                       ctx->stream));
    if ((s = take_status(ctx))) return s;
    for (int i = 0; i < n_seg; ++i)
        out[i] = cc_rp_result{h[i].max, h[i].min, h[i].argmax, h[i].argmin, h[i].count};
    return CC_OK;
}

cc_status cc_segment_extremes(cc_ctx* ctx, int32_t field_id, const cc_params* params,
                              const uint32_t* pa, const uint32_t* pb, int pairs_on_device,
                              const int64_t* seg_offsets, int n_seg, float* values,
                              cc_rp_result* out) {
    return cc_segment_extremes2(ctx, field_id, field_id, params, pa, pb, pairs_on_device,
                                seg_offsets, n_seg, values, out);
}

cc_status cc_all_pairs(cc_ctx* ctx, int32_t region_a, int32_t region_b, const cc_params* params,
                       float* values, int64_t ld, cc_rp_result* out) {
    if (!ctx) return CC_ERR_INVALID_ARG;
    Region* ra = get_region(ctx, region_a);
    Region* rb = get_region(ctx, region_b);
    if (!ra || !rb || !out) return fail(ctx, CC_ERR_INVALID_ARG, "bad arguments");
    Field& fa = *ctx->fields[ra->field];
    Field& fb = *ctx->fields[rb->field];
    if (fa.n != fb.n) return fail(ctx, CC_ERR_INVALID_ARG, "fields differ in member count");
    cc_status s = check_params(ctx, params, fa.n, nullptr);
    if (s) return s;
    if (params->measure != CC_PEARSON && params->measure != CC_SPEARMAN)
        return fail(ctx, CC_ERR_UNSUPPORTED, "all-pairs supports Pearson and Spearman");
    if (params->precision == CC_BF16 || params->precision == CC_FP8_E4M3) {
        if (values) return fail(ctx, CC_ERR_INVALID_ARG, "reduced precision stores no values");
        return cc_all_pairs_topk(ctx, region_a, region_b, params, 0, nullptr, nullptr, out,
                                 nullptr);
    }
    if (params->precision != CC_FP32)
        return fail(ctx, CC_ERR_UNSUPPORTED, "all-pairs precision %d not built",
                    params->precision);
    if (values && ld < rb->np) return fail(ctx, CC_ERR_INVALID_ARG, "ld < |B|");
    if ((ra->np + 127) / 128 > 65535) return fail(ctx, CC_ERR_INVALID_ARG, "region too large");
    if ((s = ensure_region_planes(ctx, *ra))) return s;
    if ((s = ensure_region_planes(ctx, *rb))) return s;
    const int self = region_a == region_b;
    const size_t np = allpairs_partials(ra->np, rb->np);
    CK(ctx->partials.ensure(sizeof(Partial) * (np + 1)));
    Partial* parts = ctx->partials.as<Partial>();
    const bool sp = params->measure == CC_SPEARMAN;
    CK(launch_allpairs_f32(sp ? ra->rT.as<float>() : ra->zT.as<float>(), ra->np_pad,
                           sp ? rb->rT.as<float>() : rb->zT.as<float>(), rb->np_pad, ra->nk,
                           ra->np, rb->np, self, values, ld, parts, parts + np, ctx->stream));
    Partial h;
    CK(cudaMemcpyAsync(&h, parts + np, sizeof(Partial), cudaMemcpyDeviceToHost, ctx->stream));
    if ((s = take_status(ctx))) return s;
    *out = cc_rp_result{h.max, h.min, h.argmax, h.argmin, h.count};
    return CC_OK;
}

}  // extern "C"

namespace {

// Reduced-precision plane of a region (rows padded to 256, K to 128 bytes).
// BF16 Spearman with n <= 257 contracts the integer centred ranks exactly
// (see k_quantize_ranks); the approximate values then differ from the exact
// ones only by the epilogue's two fp32 scalings.
bool rank_exact(bool sp, bool fp8, int n) { return sp && !fp8 && n <= 257; }

// Replay the graph cached under `key`, or capture `enqueue` on the context's
// stream into a new one (relaxed capture: the launchers may set function
// attributes), keep it (at most 16 per cache, the oldest dropped) and launch
// it. The library's launch counter counts the captured kernels once per run.
template <class F>
cudaError_t run_cached_graph(cc_ctx* ctx, std::vector<cc_ctx::CachedGraph>& cache,
                             const std::vector<uint64_t>& key, F&& enqueue) {
    cudaStream_t st = ctx->stream;
    for (auto& g : cache)
        if (g.key == key) {
            note_launch(g.kernels);
            return cudaGraphLaunch(g.exec, st);
        }
    const uint64_t before = g_launches.load();
    cudaError_t e = cudaStreamBeginCapture(st, cudaStreamCaptureModeRelaxed);
    if (e != cudaSuccess) return e;
    const cudaError_t e_run = enqueue();
    cudaGraph_t graph = nullptr;
    e = cudaStreamEndCapture(st, &graph);
    const int kernels = (int)(g_launches.load() - before);
    g_launches.fetch_sub((uint64_t)kernels);
    if (e_run != cudaSuccess || e != cudaSuccess) {
        if (graph) cudaGraphDestroy(graph);
        return e_run != cudaSuccess ? e_run : e;
    }
    cudaGraphExec_t exec = nullptr;
    e = cudaGraphInstantiate(&exec, graph, 0);
    cudaGraphDestroy(graph);
    if (e != cudaSuccess) return e;
    if (cache.size() >= 16) {
        cudaGraphExecDestroy(cache.front().exec);
        cache.erase(cache.begin());
    }
    cache.push_back({key, exec, kernels});
    note_launch(kernels);
    return cudaGraphLaunch(exec, st);
}

cc_status ensure_qplane(cc_ctx* ctx, Region& r, bool sp, bool fp8, Region::QPlane** out) {
    Field& f = *ctx->fields[r.field];
    auto& slot = r.qplanes[(sp ? 2 : 0) + (fp8 ? 1 : 0)];
    if (!slot) slot = std::make_unique<Region::QPlane>();
    Region::QPlane& qp = *slot;
    *out = &qp;
    if (qp.version == f.version) return CC_OK;
    if (!qp.q.p) {
        qp.rows_pad = (r.np + 255) / 256 * 256;
        qp.kbytes = fp8 ? round_up(f.n, 128) : round_up(f.n, 64) * 2;
        CK(qp.q.alloc((size_t)qp.rows_pad * qp.kbytes));
        CK(qp.inv.alloc(sizeof(float) * qp.rows_pad));
        CK(qp.emax.alloc(sizeof(unsigned)));
    }
    CK(cudaMemsetAsync(qp.emax.p, 0, sizeof(unsigned), ctx->stream));
    if (rank_exact(sp, fp8, f.n))  // integer ranks: exact operands, e_p = 0
        CK(launch_quantize_ranks(f.rank2.as<int16_t>(), f.n_pad, f.n, r.pts.as<uint32_t>(), r.np,
                                 qp.rows_pad, qp.kbytes, qp.q.p, qp.inv.as<float>(),
                                 ctx->stream));
    else
        CK(launch_quantize(fp8, sp ? f.rhat.as<float>() : f.zhat.as<float>(), f.n_pad, f.n,
                           r.pts.as<uint32_t>(), r.np, qp.rows_pad, qp.kbytes, qp.q.p,
                           qp.inv.as<float>(), qp.emax.as<unsigned>(), ctx->stream));
    qp.version = f.version;  // the error norm stays on the device (read by the threshold)
    return CC_OK;
}

float unorder_key(unsigned o) {
    unsigned b = (o & 0x80000000u) ? (o & 0x7fffffffu) : ~o;
    float v;
    memcpy(&v, &b, sizeof v);
    return v;
}

}  // namespace

extern "C" cc_status cc_all_pairs_topk(cc_ctx* ctx, int32_t region_a, int32_t region_b,
                                       const cc_params* params, int topk, uint64_t* ids,
                                       float* vals, cc_rp_result* out, cc_mixed_info* info) {
    if (!ctx) return CC_ERR_INVALID_ARG;
    Region* ra = get_region(ctx, region_a);
    Region* rb = get_region(ctx, region_b);
    if (!ra || !rb || !out) return fail(ctx, CC_ERR_INVALID_ARG, "bad arguments");
    Field& fa = *ctx->fields[ra->field];
    Field& fb = *ctx->fields[rb->field];
    if (fa.n != fb.n) return fail(ctx, CC_ERR_INVALID_ARG, "fields differ in member count");
    cc_status s = check_params(ctx, params, fa.n, nullptr);
    if (s) return s;
    if (params->measure != CC_PEARSON && params->measure != CC_SPEARMAN)
        return fail(ctx, CC_ERR_UNSUPPORTED, "reduced precision supports Pearson and Spearman");
    if (params->precision != CC_BF16 && params->precision != CC_FP8_E4M3)
        return fail(ctx, CC_ERR_INVALID_ARG, "precision must be CC_BF16 or CC_FP8_E4M3");
    if (topk < 0 || topk > 4096 || (topk > 0 && (!ids || !vals)))
        return fail(ctx, CC_ERR_INVALID_ARG, "topk in [0, 4096] with ids and vals");
    if ((uint64_t)ra->np * (uint64_t)rb->np >= (1ull << 32))
        return fail(ctx, CC_ERR_INVALID_ARG, "|A| * |B| must be below 2^32");
    const bool fp8 = params->precision == CC_FP8_E4M3, sp = params->measure == CC_SPEARMAN;
    const int self = region_a == region_b;
    Region::QPlane *qa = nullptr, *qb = nullptr;
    if ((s = ensure_qplane(ctx, *ra, sp, fp8, &qa))) return s;
    if ((s = ensure_qplane(ctx, *rb, sp, fp8, &qb))) return s;
    const int64_t na = ra->np, nb = rb->np, na_pad = qa->rows_pad, nb_pad = qb->rows_pad;
    const int64_t N = (nb_pad / 32) * na_pad;  // chunks
    const unsigned cap = 1u << 18;             // candidate chunks per extreme
    // scratch arena
    size_t off = 0;
    auto take = [&](size_t bytes) {
        const size_t o = off;
        off += (bytes + 255) / 256 * 256;
        return o;
    };
    // scratch arena; the 2 x 4096 histogram bins, the two side records and the
    // top-K selection state are contiguous so one memset clears them
    const size_t o_hist = take(4 * 2 * 4096 + sizeof(SideState) * 2 + sizeof(Select));
    const size_t o_cmax = take(4 * N), o_cmin = take(4 * N), o_ids = take(2 * 4ull * cap),
                 o_vals = take(2 * 4ull * cap * 32), o_pids = take(2 * 8ull * cap * 32),
                 o_sidx = take(4 * 8192), o_tv = take(4 * 4096), o_ti = take(8 * 4096),
                 o_sk = take(8 * 8192);
    CK(ctx->mixed.ensure(off));
    unsigned char* base = ctx->mixed.as<unsigned char>();
    float* cmax = (float*)(base + o_cmax);
    float* cmin = (float*)(base + o_cmin);
    unsigned* hist = (unsigned*)(base + o_hist);
    SideState* ss = (SideState*)(hist + 2 * 4096);
    Select* topsel = (Select*)(ss + 2);
    uint32_t* cids = (uint32_t*)(base + o_ids);
    float* rvals = (float*)(base + o_vals);
    unsigned long long* rpids = (unsigned long long*)(base + o_pids);
    uint32_t* sidx = (uint32_t*)(base + o_sidx);
    float* tvals = (float*)(base + o_tv);
    unsigned long long* tids = (unsigned long long*)(base + o_ti);
    cudaStream_t st = ctx->stream;
    const bool exact = rank_exact(sp, fp8, fa.n);
    const float* plane_a = sp ? fa.rhat.as<float>() : fa.zhat.as<float>();
    const float* plane_b = sp ? fb.rhat.as<float>() : fb.zhat.as<float>();
    // The device work below is ~20 launches; it is captured once into a CUDA
    // graph per distinct set of buffers and sizes and replayed, so the GPU
    // runs the launches back to back instead of waiting on the host. Every
    // pointer and scalar the launches take is part of the key, so a replay
    // does exactly what a fresh enqueue would.
    const std::vector<uint64_t> key = {
        (uint64_t)(uintptr_t)qa->q.p, (uint64_t)(uintptr_t)qb->q.p,
        (uint64_t)(uintptr_t)qa->inv.p, (uint64_t)(uintptr_t)qb->inv.p,
        (uint64_t)(uintptr_t)qa->emax.p, (uint64_t)(uintptr_t)qb->emax.p,
        (uint64_t)(uintptr_t)plane_a, (uint64_t)(uintptr_t)plane_b,
        (uint64_t)(uintptr_t)ra->pts.p, (uint64_t)(uintptr_t)rb->pts.p,
        (uint64_t)(uintptr_t)base, (uint64_t)(uintptr_t)ctx->status.p, (uint64_t)(uintptr_t)st,
        (uint64_t)na, (uint64_t)nb, (uint64_t)na_pad, (uint64_t)nb_pad, (uint64_t)qa->kbytes,
        (uint64_t)fa.n, (uint64_t)fa.n_pad, (uint64_t)self, (uint64_t)fp8, (uint64_t)exact,
        (uint64_t)topk};
#define EK(call)                                \
    do {                                        \
        const cudaError_t _e = (call);          \
        if (_e != cudaSuccess) return _e;       \
    } while (0)
    auto enqueue = [&]() -> cudaError_t {
        EK(cudaMemsetAsync(hist, 0, 4 * 2 * 4096 + sizeof(SideState) * 2 + sizeof(Select), st));
        // the tensor-core kernel builds the first-level selection histogram
        // when its epilogue has slack (K of 8 or more 128-byte blocks: the
        // contraction, not the epilogue, bounds it); with short K the epilogue
        // is the bound and a separate pass is faster
        const bool hist_fused = qa->kbytes / 128 >= 8;
        EK(launch_tc_chunk_extremes(fp8, fp8 || exact, qa->q.p, na, na_pad, qb->q.p, nb, nb_pad,
                                    qa->kbytes, self, qa->inv.as<float>(), qb->inv.as<float>(), cmax,
                                    cmin, hist_fused ? hist : nullptr, ctx->status.as<int>(), st));
        // relative error of the approximate values beyond the quantization error:
        // FP32 accumulation (2^-12, conservative), or for exact integer ranks the
        // two fp32 scalings of the epilogue (2^-22 covers them)
        const float acc_rel = exact ? 1.f / 4194304.f : 1.f / 4096.f;
        // Both sides (maximum: keys of cmax; minimum: keys of -cmin) share every
        // launch. Both passes are decided on the device (no host round trip):
        // the second compaction appends the chunks in [r* - B, first threshold)
        // after the first pass's, unless the first pass took every chunk or
        // overflowed.
        EK(launch_select_top2(cmax, cmin, N, (unsigned)std::max(topk, 256), 256u, hist,
                              hist_fused, ss, cids, cap, st));
        EK(launch_refine_chunks2(plane_a, plane_b, fa.n_pad, fa.n, ra->pts.as<uint32_t>(), na,
                                 rb->pts.as<uint32_t>(), nb, self, na_pad, cids, cap, ss, true,
                                 rvals, rpids, fp8, st));
        EK(launch_second_threshold2(ss, qa->emax.as<unsigned>(), qb->emax.as<unsigned>(), acc_rel,
                                    st));
        EK(launch_compact_second2(cmax, cmin, N, ss, cids, cap, st));
        EK(launch_refine_chunks2(plane_a, plane_b, fa.n_pad, fa.n, ra->pts.as<uint32_t>(), na,
                                 rb->pts.as<uint32_t>(), nb, self, na_pad, cids, cap, ss, false,
                                 rvals, rpids, fp8, st));
        if (topk > 0) {  // top-K of every refined value of the maximum side
            EK(launch_select_top(rvals, (int64_t)cap * 32, 1.f, (unsigned)topk, hist, topsel, sidx,
                                 8192, st, &ss[0].sel.count));
            EK(launch_sort_top(rvals, rpids, sidx, &topsel->count, 8192, 1.f, topk, tvals, tids,
                               (unsigned long long*)(base + o_sk), st));
        }
        return cudaSuccess;
    };
#undef EK
    CK(run_cached_graph(ctx, ctx->topk_graphs, key, enqueue));
    // the side records and the top list land in pinned memory (asynchronous
    // copies, one wait) and are copied out on the host
    SideState hout[2];
    const size_t o_hv = 256, o_hi = o_hv + 4 * (size_t)topk;
    CK(ctx->host_out.ensure(o_hi + 8 * (size_t)topk));
    unsigned char* hb = ctx->host_out.as<unsigned char>();
    static_assert(sizeof(SideState) * 2 + sizeof(int) <= 256, "landing area");
    CK(cudaMemcpyAsync(hb, ss, sizeof hout, cudaMemcpyDeviceToHost, st));
    CK(cudaMemcpyAsync(hb + sizeof hout, ctx->status.p, sizeof(int), cudaMemcpyDeviceToHost, st));
    if (topk > 0) {
        CK(cudaMemcpyAsync(hb + o_hv, tvals, 4 * (size_t)topk, cudaMemcpyDeviceToHost, st));
        CK(cudaMemcpyAsync(hb + o_hi, tids, 8 * (size_t)topk, cudaMemcpyDeviceToHost, st));
    }
    CK(cudaStreamSynchronize(st));
    memcpy(hout, hb, sizeof hout);
    int dev_status = 0;
    memcpy(&dev_status, hb + sizeof hout, sizeof(int));
    if (topk > 0) {
        memcpy(vals, hb + o_hv, 4 * (size_t)topk);
        memcpy(ids, hb + o_hi, 8 * (size_t)topk);
    }
    if ((s = status_value(ctx, dev_status))) return s;
    cc_mixed_info inf{};
    float ext_val[2] = {-INFINITY, -INFINITY};
    uint64_t ext_id[2] = {~0ull, ~0ull};
    for (int side = 0; side < 2; ++side) {
        const SideState& o = hout[side];
        const bool certified = o.sel.overflow == 0;  // both passes fit (or pass 1 took all)
        if (o.best != 0) {
            ext_val[side] = unorder_key((unsigned)(o.best >> 32));
            ext_id[side] = 0xffffffffull - (o.best & 0xffffffffull);
        }
        inf.bound = o.thr[1];
        if (side == 0) {
            inf.threshold_max = o.thr[0];
            inf.certified_max = certified;
        } else {
            inf.threshold_min = -o.thr[0];
            inf.certified_min = certified;
        }
        inf.refined_pairs += (int64_t)std::min(o.sel.count, cap) * 32;
    }
    const uint64_t count = self ? (uint64_t)na * (na - 1) / 2 : (uint64_t)na * nb;
    *out = cc_rp_result{ext_val[0], -ext_val[1], ext_id[0], ext_id[1], count};
    if (info) *info = inf;
    return CC_OK;
}

extern "C" cc_status cc_all_pairs_approx(cc_ctx* ctx, int32_t region_a, int32_t region_b,
                                         const cc_params* params, float* cmax, float* cmin,
                                         float* bound) {
    if (!ctx) return CC_ERR_INVALID_ARG;
    Region* ra = get_region(ctx, region_a);
    Region* rb = get_region(ctx, region_b);
    if (!ra || !rb || !cmax || !cmin || !bound) return fail(ctx, CC_ERR_INVALID_ARG, "bad arguments");
    Field& fa = *ctx->fields[ra->field];
    Field& fb = *ctx->fields[rb->field];
    if (fa.n != fb.n) return fail(ctx, CC_ERR_INVALID_ARG, "fields differ in member count");
    cc_status s = check_params(ctx, params, fa.n, nullptr);
    if (s) return s;
    if (params->measure != CC_PEARSON && params->measure != CC_SPEARMAN)
        return fail(ctx, CC_ERR_UNSUPPORTED, "reduced precision supports Pearson and Spearman");
    if (params->precision != CC_BF16 && params->precision != CC_FP8_E4M3)
        return fail(ctx, CC_ERR_INVALID_ARG, "precision must be CC_BF16 or CC_FP8_E4M3");
    const bool fp8 = params->precision == CC_FP8_E4M3, sp = params->measure == CC_SPEARMAN;
    const int self = region_a == region_b;
    Region::QPlane *qa = nullptr, *qb = nullptr;
    if ((s = ensure_qplane(ctx, *ra, sp, fp8, &qa))) return s;
    if ((s = ensure_qplane(ctx, *rb, sp, fp8, &qb))) return s;
    const int64_t na = ra->np, nb = rb->np, na_pad = qa->rows_pad, nb_pad = qb->rows_pad;
    const int64_t N = (nb_pad / 32) * na_pad, chunks = (nb + 31) / 32;
    CK(ctx->approx.ensure(8 * (size_t)N + 16));
    float* dmax = ctx->approx.as<float>();
    float* dmin = dmax + N;
    unsigned* demax = reinterpret_cast<unsigned*>(dmin + N);
    cudaStream_t st = ctx->stream;
    const bool exact = rank_exact(sp, fp8, fa.n);
    CK(launch_tc_chunk_extremes(fp8, fp8 || exact, qa->q.p, na, na_pad, qb->q.p, nb, nb_pad,
                                qa->kbytes, self, qa->inv.as<float>(), qb->inv.as<float>(), dmax,
                                dmin, nullptr, ctx->status.as<int>(), st));
    CK(cudaMemcpyAsync(demax, qa->emax.p, 4, cudaMemcpyDeviceToDevice, st));
    CK(cudaMemcpyAsync(demax + 1, qb->emax.p, 4, cudaMemcpyDeviceToDevice, st));
    CK(cudaMemcpy2DAsync(cmax, sizeof(float) * na, dmax, sizeof(float) * na_pad,
                         sizeof(float) * na, chunks, cudaMemcpyDeviceToHost, st));
    CK(cudaMemcpy2DAsync(cmin, sizeof(float) * na, dmin, sizeof(float) * na_pad,
                         sizeof(float) * na, chunks, cudaMemcpyDeviceToHost, st));
    unsigned eb[2] = {0, 0};
    CK(cudaMemcpyAsync(eb, demax, 8, cudaMemcpyDeviceToHost, st));
    CK(cudaStreamSynchronize(st));
    if ((s = take_status(ctx))) return s;
    // the bound of the certified path (cc_all_pairs_topk), same arithmetic
    float ea, eb2;
    memcpy(&ea, &eb[0], 4);
    memcpy(&eb2, &eb[1], 4);
    const float e = exact ? 0.f : std::max(ea, eb2);
    const float acc_rel = exact ? 1.f / 4194304.f : 1.f / 4096.f;
    *bound = 2.f * e + e * e + (1.f + e) * (1.f + e) * acc_rel + 1e-6f;
    return CC_OK;
}
