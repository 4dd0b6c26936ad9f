// abi_common.h -- internals shared by the C ABI translation units: the
// context, status helpers, argument validation, library-owned scratch and
// the kernel argument block of one problem.
#pragma once

#include <algorithm>
#include <climits>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <functional>
#include <mutex>
#include <new>
#include <vector>

#include <cuda.h>
#include <cudaTypedefs.h>

#include "flamerec.h"
#include "fr_internal.h"

using namespace frk;

struct Buf {
    void* p = nullptr;
    size_t bytes = 0;
};

constexpr size_t kHostScratchBytes = 64;

// Forward and adjustment of an iteration pipelined view by view over two
// streams (fr_reconstruct) when 1; 0 (the default) launches each once over all
// views (the pipelined form measured 1.19 ms against 0.714 ms per iteration of
// the full-RTE workload).
#ifndef FR_NODE_BOX
#define FR_NODE_BOX 1
#endif
#ifndef FR_SPLIT_BOX
#define FR_SPLIT_BOX 1
#endif
#ifndef FR_SWEEP_PACK
#define FR_SWEEP_PACK 1
#endif
// FR_LIST_DL = 1: in the loop over all views, the forward stores each flame
// ray's residual beside its list entries and writes no residual image (the
// adjustment 0.278 against 0.280 ms)
#ifndef FR_LIST_DL
#define FR_LIST_DL 1
#endif
#ifndef FR_PIPELINE_VIEWS
#define FR_PIPELINE_VIEWS 0
#endif

struct fr_ctx {
    int device = 0;
    cudaStream_t stream = nullptr;   // where work is queued (borrowed; 0 = default stream)
    char err[512] = {0};             // last failure message
    Buf partials, counter, residual, rendered, dV, targets, sqerr, rmse, J, src, flame_cnt, flame_list;
    Buf batch;                       // batched reconstruction scratch and tables
    Buf pairs;                       // x-pair records for the forward march
    Buf occ;                         // brick occupancy for empty-space skipping
    Buf hull_bricks;                 // bricks holding a key point inside the visual hull
    Buf loop;                        // device iteration counter of fr_reconstruct_until
    Buf fin;                         // multi-CTA error reduction: part sums and its counter (kept 0)
    Buf flame_tm;                    // transmittance at the split of each listed flame ray's second half
    Buf flame_dl;                    // residual of each listed flame ray (FR_LIST_DL)
    // dV holds zeros over its first dV_zero_bytes when dV.p == dV_zero_at: a
    // completed reconstruction leaves it so (each update zeroes what it adds)
    const void* dV_zero_at = nullptr;
    size_t dV_zero_bytes = 0;
    Buf verr;                        // volume-error partials and result
    Buf L6;                          // directional radiances for anisotropic in-scattering
    Buf hull, sat;                   // visual hull tags, flame-mask tables
    Buf vol_stage;                   // float32 staging of fr_volume_upload / fr_volume_download
    Buf probe;                       // measurement builds only (FR_ADJ_GATHER_PROBE)
    Buf tab_small, tab_fwd;          // ray weight tables: counts, offsets and the hull's list; the tables
    std::vector<Buf> tab_batch;      // the same per problem of fr_reconstruct_batch (two each)
    Buf torder;                      // marching loop: the forward's tile keys and launch order
    unsigned long long tab_stats[4] = {0, 0, 0, 0};  // sizes of the last call's tables (fr_table_stats)
    void* tab_host = nullptr;        // pinned host scratch of the tables' build (warps' rows, tile order)
    size_t tab_host_bytes = 0;
    std::vector<void*> owned;        // volume records allocated by fr_volume_create
    unsigned long long* host_counter = nullptr;  // pinned host scratch of kHostScratchBytes
    void* staging = nullptr;         // pinned host staging of batch tables
    size_t staging_bytes = 0;
    cudaEvent_t staging_done = nullptr;
    cudaStream_t capture = nullptr;  // stream used to capture CUDA graphs
    cudaStream_t aux = nullptr;      // second stream of the pipelined views (adjustments)
    cudaEvent_t pipe_ev[kMaxViews + 1] = {};  // per-view forward done; [kMaxViews]: adjustments done
    // device scratch held in Bufs, and the most the context may hold
    size_t scratch_bytes = 0;
    size_t scratch_limit = SIZE_MAX;
    // phase tracing: events recorded between the phases of fr_reconstruct
    bool trace_on = false;
    bool trace_overflow = false;
    std::vector<cudaEvent_t> trace_pool;          // created on demand, reused
    std::vector<int> trace_phase;                 // phase of the interval ending at event i (-1: none)
};

namespace frabi {

inline fr_status fail(fr_ctx* c, fr_status s, const char* fmt, ...)
{
    if (c) {
        va_list ap;
        va_start(ap, fmt);
        vsnprintf(c->err, sizeof c->err, fmt, ap);
        va_end(ap);
    }
    return s;
}

inline fr_status cuda_fail(fr_ctx* c, cudaError_t e, const char* what)
{
    return fail(c, FR_ECUDA, "%s: %s (%s)", what, cudaGetErrorName(e), cudaGetErrorString(e));
}

#define FR_CUDA(ctx, expr)                                 \
    do {                                                   \
        cudaError_t e_ = (expr);                           \
        if (e_ != cudaSuccess) return cuda_fail(ctx, e_, #expr); \
    } while (0)

// Device-pointer check: the pointer must lie in a device allocation that
// holds at least `bytes` from it.  Catches host pointers and short buffers
// before any kernel could touch them.
inline PFN_cuMemGetAddressRange_v3020 range_fn()
{
    static PFN_cuMemGetAddressRange_v3020 fn = nullptr;
    static std::once_flag once;
    std::call_once(once, [] {
        void* f = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuMemGetAddressRange", &f, 12000, cudaEnableDefault, &q) ==
                cudaSuccess && q == cudaDriverEntryPointSuccess)
            fn = reinterpret_cast<PFN_cuMemGetAddressRange_v3020>(f);
    });
    return fn;
}

inline fr_status check_dev(fr_ctx* c, const void* p, size_t bytes, const char* name)
{
    if (!p) return fail(c, FR_EINVAL, "%s is NULL", name);
    cudaPointerAttributes at;
    cudaError_t e = cudaPointerGetAttributes(&at, p);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return fail(c, FR_EINVAL, "%s is not a CUDA pointer (%s)", name, cudaGetErrorName(e));
    }
    if (at.type != cudaMemoryTypeDevice && at.type != cudaMemoryTypeManaged)
        return fail(c, FR_EINVAL, "%s must be device memory", name);
    if (at.type == cudaMemoryTypeDevice && at.device != c->device)
        return fail(c, FR_EINVAL, "%s lives on device %d, context on %d", name, at.device, c->device);
    if (auto fn = range_fn()) {
        CUdeviceptr base = 0;
        size_t size = 0;
        if (fn(&base, &size, (CUdeviceptr)(uintptr_t)p) == CUDA_SUCCESS) {
            if ((uintptr_t)p + bytes > (uintptr_t)base + size)
                return fail(c, FR_EINVAL, "%s: %zu bytes needed but the allocation ends %zu bytes after it",
                            name, bytes, (size_t)((uintptr_t)base + size - (uintptr_t)p));
        }
    }
    return FR_OK;
}

inline fr_status check_align(fr_ctx* c, const void* p, size_t a, const char* name)
{
    if ((uintptr_t)p % a) return fail(c, FR_EINVAL, "%s must be %zu-byte aligned", name, a);
    return FR_OK;
}

inline int rec_components(int kind) { return kind == FR_KIND_RGB ? 4 : 2; }
inline int dtype_bytes(int dt) { return dt == FR_F32 ? 4 : 2; }
inline size_t rec_bytes(const fr_volume* v) { return (size_t)rec_components(v->kind) * dtype_bytes(v->dtype); }
inline long long node_count(const fr_volume* v) { return (long long)v->nx * v->ny * v->nz; }

inline bool finite3(const float* x) { return std::isfinite(x[0]) && std::isfinite(x[1]) && std::isfinite(x[2]); }

inline fr_status check_volume(fr_ctx* c, const fr_volume* v, const char* name)
{
    if (!v) return fail(c, FR_EINVAL, "%s is NULL", name);
    if (v->nx < 2 || v->ny < 2 || v->nz < 2 || v->nx > 8192 || v->ny > 8192 || v->nz > 8192)
        return fail(c, FR_EINVAL, "%s: extents must be in [2, 8192], got %d x %d x %d", name, v->nx, v->ny, v->nz);
    if (node_count(v) >= (1LL << 31)) return fail(c, FR_EINVAL, "%s: at most 2^31 - 1 nodes", name);
    if (v->kind != FR_KIND_RGB && v->kind != FR_KIND_TEMP) return fail(c, FR_EINVAL, "%s: bad kind %d", name, v->kind);
    if (v->dtype != FR_F32 && v->dtype != FR_BF16 && v->dtype != FR_F16)
        return fail(c, FR_EINVAL, "%s: bad dtype %d", name, v->dtype);
    if (!(v->h > 0.0f) || !std::isfinite(v->h) || !finite3(v->origin))
        return fail(c, FR_EINVAL, "%s: spacing must be positive and origin finite", name);
    fr_status s = check_align(c, v->data, rec_bytes(v), name);
    if (s) return s;
    return check_dev(c, v->data, (size_t)node_count(v) * rec_bytes(v), name);
}

inline fr_status check_cams(fr_ctx* c, const fr_camera* cams, int ncam)
{
    if (!cams) return fail(c, FR_EINVAL, "cams is NULL");
    if (ncam < 1 || ncam > kMaxViews) return fail(c, FR_EINVAL, "ncam must be in [1, %d], got %d", kMaxViews, ncam);
    for (int i = 0; i < ncam; ++i) {
        const fr_camera& k = cams[i];
        if (k.width < 1 || k.height < 1 || k.width > 16384 || k.height > 16384)
            return fail(c, FR_EINVAL, "camera %d: image size must be in [1, 16384]", i);
        if (k.width != cams[0].width || k.height != cams[0].height)
            return fail(c, FR_EINVAL, "camera %d: all cameras must share one image size", i);
        if (!(k.tan_half_fov > 0.0f) || !std::isfinite(k.tan_half_fov))
            return fail(c, FR_EINVAL, "camera %d: tan_half_fov must be positive", i);
        if (!finite3(k.pos) || !finite3(k.right) || !finite3(k.up) || !finite3(k.fwd))
            return fail(c, FR_EINVAL, "camera %d: non-finite vector", i);
        auto dot = [](const float* a, const float* b) { return a[0] * b[0] + a[1] * b[1] + a[2] * b[2]; };
        if (fabsf(dot(k.fwd, k.fwd) - 1.0f) > 1e-3f || fabsf(dot(k.right, k.right) - 1.0f) > 1e-3f ||
            fabsf(dot(k.up, k.up) - 1.0f) > 1e-3f || fabsf(dot(k.fwd, k.right)) > 1e-3f ||
            fabsf(dot(k.fwd, k.up)) > 1e-3f || fabsf(dot(k.right, k.up)) > 1e-3f)
            return fail(c, FR_EINVAL, "camera %d: right, up, fwd must be orthonormal", i);
    }
    return FR_OK;
}

inline fr_status check_params(fr_ctx* c, const fr_params* p, const fr_volume* v, const fr_camera* cams)
{
    if (!p) return fail(c, FR_EINVAL, "params is NULL");
    if (!(p->step > 0.0f) || !std::isfinite(p->step)) return fail(c, FR_EINVAL, "step must be positive");
    double diag = std::sqrt((double)(v->nx - 1) * (v->nx - 1) + (double)(v->ny - 1) * (v->ny - 1) +
                            (double)(v->nz - 1) * (v->nz - 1));
    double max_seg = std::ceil(diag / p->step) + 1.0;
    if (max_seg > 1e6) return fail(c, FR_EINVAL, "step too small: up to %.0f samples per ray", max_seg);
    if (!std::isfinite(p->alpha_l) || !std::isfinite(p->alpha_d) || p->alpha_d < 0.0f)
        return fail(c, FR_EINVAL, "alpha_l must be finite and alpha_d finite and >= 0");
    if (!(p->tau < 1.0f) || !std::isfinite(p->tau)) return fail(c, FR_EINVAL, "tau must be < 1");
    if (!std::isfinite(p->flame_thresh)) return fail(c, FR_EINVAL, "flame_thresh must be finite");
    if (!(p->g_std >= 0.0f) || !std::isfinite(p->g_std)) return fail(c, FR_EINVAL, "g_std must be >= 0");
    if (p->g_std > 0.0f) {
        // counter layout of the G(s) stream: 20 bits iteration, 8 view, 22 pixel, 14 sample
        if ((long long)cams[0].width * cams[0].height > (1LL << 22))
            return fail(c, FR_EINVAL, "g_std > 0 supports at most 2^22 pixels per view");
        if (max_seg > 16383.0) return fail(c, FR_EINVAL, "g_std > 0 supports at most 16383 samples per ray");
    }
    if (v->kind == FR_KIND_TEMP) {
        if (!p->lut || p->lut_size < 2 || !(p->lut_t_max > p->lut_t_min))
            return fail(c, FR_EINVAL, "temperature volumes need lut, lut_size >= 2 and lut_t_max > lut_t_min");
        fr_status s = check_align(c, p->lut, 16, "lut");
        if (s) return s;
        return check_dev(c, p->lut, (size_t)p->lut_size * 16, "lut");
    }
    return FR_OK;
}

inline fr_status ensure(fr_ctx* c, Buf& b, size_t bytes, const char* name)
{
    if (b.bytes >= bytes) return FR_OK;
    size_t want = bytes < 256 ? 256 : bytes;
    if (c->scratch_bytes - b.bytes + want > c->scratch_limit)
        return fail(c, FR_ENOMEM, "%s scratch of %zu bytes would exceed the context's limit of %zu bytes", name,
                    want, c->scratch_limit);
    if (b.p) {
        FR_CUDA(c, cudaStreamSynchronize(c->stream));
        cudaFree(b.p);
        c->scratch_bytes -= b.bytes;
        b.p = nullptr;
        b.bytes = 0;
    }
    cudaError_t e = cudaMalloc(&b.p, want);
    if (e != cudaSuccess) {
        cudaGetLastError();
        b.p = nullptr;
        return fail(c, FR_ENOMEM, "cannot allocate %zu bytes of %s scratch", want, name);
    }
    b.bytes = want;
    c->scratch_bytes += want;
    return FR_OK;
}

inline void fill_problem(const fr_volume* v, const fr_camera* cams, int ncam, const fr_params* p, SingleArgs& a)
{
    memset(&a, 0, sizeof a);
    ProbDev& P = a.p;
    P.vol = v->data;
    P.nx = v->nx; P.ny = v->ny; P.nz = v->nz;
    P.ncam = ncam;
    P.W = cams[0].width;
    P.H = cams[0].height;
    P.tiles_x = (P.W + kTileW - 1) / kTileW;
    P.tiles_y = (P.H + kTileH - 1) / kTileH;
    P.img_scale = 1.0f;
    P.step = p->step;
    P.alpha_l = p->alpha_l;
    P.alpha_d = p->alpha_d;
    P.tau = p->tau > 0.0f ? p->tau : 0.0f;
    P.g_std = p->g_std;
    P.thresh = p->flame_thresh;
    P.seed = p->seed;
    if (v->kind == FR_KIND_TEMP) {
        P.lut = reinterpret_cast<const float4*>(p->lut);
        P.lut_m = p->lut_size;
        P.lut_t0 = p->lut_t_min;
        P.lut_scale = (float)(p->lut_size - 1) / (p->lut_t_max - p->lut_t_min);
    }
    const float inv_h = 1.0f / v->h;
    for (int i = 0; i < ncam; ++i) {
        CamDev& d = a.cams[i];
        const fr_camera& k = cams[i];
        for (int ax = 0; ax < 3; ++ax) {
            d.o[ax] = (k.pos[ax] - v->origin[ax]) * inv_h;
            d.r[ax] = k.right[ax];
            d.u[ax] = k.up[ax];
            d.f[ax] = k.fwd[ax];
        }
        d.ty = k.tan_half_fov;
        d.tx = k.tan_half_fov * (float)k.width / (float)k.height;
        d.W = k.width;
        d.H = k.height;
    }
}

inline size_t image_bytes(const fr_camera* cams, int ncam)
{
    return (size_t)ncam * cams[0].width * cams[0].height * 3 * sizeof(float);
}

constexpr size_t kTraceMaxEvents = 1 << 16;

// Ends the interval of `phase` (-1: an interval that is not counted) with an
// event on the context's stream, when tracing is on.  Past kTraceMaxEvents
// unread events, marks are dropped and the overflow is reported on reading.
inline fr_status trace_mark(fr_ctx* c, int phase)
{
    if (!c->trace_on) return FR_OK;
    const size_t i = c->trace_phase.size();
    if (i >= kTraceMaxEvents) {
        c->trace_overflow = true;
        return FR_OK;
    }
    if (i == c->trace_pool.size()) {
        cudaEvent_t e;
        FR_CUDA(c, cudaEventCreate(&e));
        c->trace_pool.push_back(e);
    }
    FR_CUDA(c, cudaEventRecord(c->trace_pool[i], c->stream));
    c->trace_phase.push_back(phase);
    return FR_OK;
}

}  // namespace frabi

using namespace frabi;

#define FR_TRY(expr)                  \
    do {                              \
        fr_status s_ = (expr);        \
        if (s_ != FR_OK) return s_;   \
    } while (0)

#define FR_BEGIN(c)                                   \
    if (!c) return FR_EINVAL;                         \
    c->err[0] = '\0';                                 \
    FR_CUDA(c, cudaSetDevice(c->device))

inline size_t align256(size_t x) { return (x + 255) & ~(size_t)255; }

// Visual hull tags of one problem (api.cu): flame-mask tables in the
// context's scratch, one tag per node into `tags` (device).
fr_status hull_tags(fr_ctx* c, const SingleArgs& a, const float* targets, float thresh, unsigned* tags);

// Where build_tables takes its device memory: `scratch` (counts, offsets and
// the hull's list, used by every iteration too) and then `tables` (the two
// tables, the flame rays' residuals and the hull's staged records in one
// block); either returns nullptr when there is no room (the caller then
// marches) and sets *status to another code than FR_ENOMEM on a real error.
struct TabMemory {
    std::function<void*(size_t)> scratch, tables;
    fr_status* status = nullptr;
};

// The ray weight tables of one problem (api.cu): f the problem (cameras,
// targets) with the hull's brick table (adj_occ, adj_box) and its
// parameters; vol the volume whose extinction fixes the transmittance.
// built = false (and FR_OK) when there was no room or the tables would need
// 2^32 entries; *bytes: the device bytes taken from `mem`.
fr_status build_tables(fr_ctx* c, const SingleArgs& f, const fr_volume* vol, const unsigned* tags, unsigned full,
                       int nt, const TabMemory& mem, TabIter& it, bool& built, size_t* bytes = nullptr);
