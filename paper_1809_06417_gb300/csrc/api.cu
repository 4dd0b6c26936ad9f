// api.cu -- the C ABI declared in include/flamerec.h: argument validation,
// library-owned scratch, kernel launches and the reconstruction loop.
#include <string>

#include "abi_common.h"

// ---------------------------------------------------------------------------
// Context
// ---------------------------------------------------------------------------

extern "C" int32_t fr_abi_version(void) { return FR_ABI_VERSION; }

extern "C" void fr_params_default(fr_params* p)
{
    if (!p) return;
    memset(p, 0, sizeof *p);
    p->step = 1.0f;
    p->alpha_l = 0.001f;
    p->alpha_d = 1.0f;
    p->tau = 0.0f;
    p->g_std = 0.0f;
    p->flame_thresh = 30.0f / 255.0f;
    p->seed = 0;
    p->clamp_nonneg = 1;
    p->rule = FR_RULE_PAPER;
    p->grad_step = 0.0f;
    p->update_sigma = 0;
    p->lut_t_min = 800.0f;
    p->lut_t_max = 2000.0f;
    p->lut = nullptr;
    p->lut_size = 0;
    p->use_hull = 0;
    p->skip_empty = 1;
}

extern "C" fr_status fr_create(fr_ctx** out, int device, void* stream)
{
    if (!out) return FR_EINVAL;
    *out = nullptr;
    int n = 0;
    if (cudaGetDeviceCount(&n) != cudaSuccess || n < 1) {
        cudaGetLastError();
        return FR_ECUDA;
    }
    if (device < 0 || device >= n) return FR_EINVAL;
    fr_ctx* c = new (std::nothrow) fr_ctx();
    if (!c) return FR_ENOMEM;
    c->device = device;
    if (cudaSetDevice(device) != cudaSuccess ||
        cudaMallocHost(&c->host_counter, kHostScratchBytes) != cudaSuccess) {
        cudaGetLastError();
        delete c;
        return FR_ECUDA;
    }
    c->stream = static_cast<cudaStream_t>(stream);
    *out = c;
    return FR_OK;
}

extern "C" fr_status fr_destroy(fr_ctx* c)
{
    if (!c) return FR_EINVAL;
    cudaSetDevice(c->device);
    cudaStreamSynchronize(c->stream);
    if (c->aux) cudaStreamSynchronize(c->aux);   // (adjustments of pipelined views)
    for (Buf* b : {&c->partials, &c->counter, &c->residual, &c->rendered, &c->dV, &c->targets, &c->sqerr,
                   &c->rmse, &c->J, &c->src, &c->flame_cnt, &c->flame_list, &c->batch, &c->pairs,
                   &c->hull, &c->sat, &c->occ, &c->hull_bricks, &c->loop, &c->verr, &c->L6, &c->fin, &c->flame_tm,
                   &c->vol_stage, &c->probe, &c->flame_dl, &c->tab_small, &c->tab_fwd, &c->torder})
        if (b->p) cudaFree(b->p);
    for (Buf& b : c->tab_batch)
        if (b.p) cudaFree(b.p);
    for (void* p : c->owned) cudaFree(p);
    if (c->host_counter) cudaFreeHost(c->host_counter);
    if (c->staging) cudaFreeHost(c->staging);
    if (c->tab_host) cudaFreeHost(c->tab_host);
    if (c->staging_done) cudaEventDestroy(c->staging_done);
    if (c->capture) cudaStreamDestroy(c->capture);
    if (c->aux) cudaStreamDestroy(c->aux);
    for (cudaEvent_t e : c->pipe_ev)
        if (e) cudaEventDestroy(e);
    for (cudaEvent_t e : c->trace_pool) cudaEventDestroy(e);
    delete c;
    return FR_OK;
}

extern "C" int32_t fr_checks_enabled(void)
{
#ifdef FR_CHECKED
    return 1;
#else
    return 0;
#endif
}

extern "C" int32_t fr_brick_cells(void) { return kBrick; }

extern "C" fr_status fr_check_word(fr_ctx* c, uint32_t* word, int reset)
{
    FR_BEGIN(c);
    if (!word) return fail(c, FR_EINVAL, "word is NULL");
    FR_CUDA(c, cudaStreamSynchronize(c->stream));
    unsigned a = 0, b = 0;
    FR_CUDA(c, check_word_march(&a, reset != 0));
    FR_CUDA(c, check_word_volume(&b, reset != 0));
    unsigned t = 0;
    FR_CUDA(c, check_word_tables(&t, reset != 0));
    *word = a | b | t;
    return FR_OK;
}

extern "C" fr_status fr_set_scratch_limit(fr_ctx* c, size_t bytes)
{
    if (!c) return FR_EINVAL;
    c->scratch_limit = bytes ? bytes : SIZE_MAX;
    return FR_OK;
}

extern "C" fr_status fr_scratch_bytes(const fr_ctx* c, size_t* held)
{
    if (!c || !held) return FR_EINVAL;
    *held = c->scratch_bytes;
    return FR_OK;
}

extern "C" fr_status fr_set_stream(fr_ctx* c, void* stream)
{
    if (!c) return FR_EINVAL;
    c->stream = static_cast<cudaStream_t>(stream);
    return FR_OK;
}

extern "C" const char* fr_last_error(const fr_ctx* c) { return c ? c->err : "null context"; }

extern "C" fr_status fr_synchronize(fr_ctx* c)
{
    if (!c) return FR_EINVAL;
    FR_CUDA(c, cudaStreamSynchronize(c->stream));
    if (c->aux) FR_CUDA(c, cudaStreamSynchronize(c->aux));
    return FR_OK;
}

// ---------------------------------------------------------------------------
// Single calls
// ---------------------------------------------------------------------------

// Whether the forward march may skip empty bricks (RGB records in field mode).
static bool skips_empty(const fr_volume* vol, const fr_params* p)
{
    return vol->kind == FR_KIND_RGB && p->skip_empty && !(p->tau > 0.0f);
}

// Scratch of the multi-CTA error reduction, its counter zeroed once.
static fr_status fin_scratch(fr_ctx* c, void** out)
{
    if (!c->fin.p) {
        FR_TRY(ensure(c, c->fin, kFinScratchBytes, "error reduction"));
        FR_CUDA(c, cudaMemsetAsync(c->fin.p, 0, kFinScratchBytes, c->stream));
    }
    *out = c->fin.p;
    return FR_OK;
}

// x-pair copy of the records the forward march will read, and (when it skips
// empty bricks) the occupancy of their bricks (library scratch).
static fr_status attach_pairs(fr_ctx* c, const fr_volume* vol, const fr_params* p, const void* records,
                              SingleArgs& a)
{
    FR_TRY(ensure(c, c->pairs, (size_t)node_count(vol) * 2 * rec_bytes(vol), "pairs"));
    const int nbx = bricks_along(vol->nx), nby = bricks_along(vol->ny), nbz = bricks_along(vol->nz);
    unsigned char* occ = nullptr;
    if (skips_empty(vol, p)) {
        FR_TRY(ensure(c, c->occ, brick_table_bytes(vol->nx, vol->ny, vol->nz), "brick occupancy"));
        occ = static_cast<unsigned char*>(c->occ.p);
    }
    FR_CUDA(c, launch_pair_pack(records, c->pairs.p, vol->dtype, vol->kind, vol->nx, vol->ny, vol->nz, occ,
                                c->stream));
    a.p.pairs = c->pairs.p;
    a.p.occ = occ;
    a.p.occ_box = occ ? brick_box(occ, nbx, nby, nbz) : nullptr;
    a.p.nbx = nbx;
    a.p.nby = nby;
    a.p.nbz = nbz;
    return FR_OK;
}

extern "C" fr_status fr_prepare_targets(fr_ctx* c, int ncam, int height, int width, float* targets,
                                        float thresh, int32_t* bbox)
{
    FR_BEGIN(c);
    if (ncam < 1 || ncam > kMaxViews || height < 1 || width < 1 || height > 16384 || width > 16384)
        return fail(c, FR_EINVAL, "bad image extents");
    if (!std::isfinite(thresh)) return fail(c, FR_EINVAL, "thresh must be finite");
    FR_TRY(check_dev(c, targets, (size_t)ncam * height * width * 3 * sizeof(float), "targets"));
    FR_TRY(check_dev(c, bbox, (size_t)ncam * 4 * sizeof(int32_t), "bbox"));
    FR_CUDA(c, launch_prepare_targets(targets, ncam, height, width, thresh, bbox, c->stream));
    return FR_OK;
}

// Large single renders take their tiles longest first (the most samples a
// ray of the tile takes through the box; brick skipping not counted).
constexpr int kOrderMinTiles = 1024;
static fr_status order_tiles(fr_ctx* c, SingleArgs& a, int nt)
{
    if (!FR_MARCH_ORDER || nt < kOrderMinTiles) return FR_OK;
    FR_TRY(ensure(c, c->torder, (size_t)nt * 8, "tile order"));
    unsigned* key = static_cast<unsigned*>(c->torder.p);
    FR_CUDA(c, launch_tile_order(a, nt, nullptr, key, key + nt, c->stream));
    a.p.tile_order = key + nt;
    return FR_OK;
}

extern "C" fr_status fr_render(fr_ctx* c, const fr_volume* vol, const fr_camera* cams, int ncam,
                               const fr_params* p, float* out_rgb)
{
    FR_BEGIN(c);
    FR_TRY(check_volume(c, vol, "vol"));
    FR_TRY(check_cams(c, cams, ncam));
    FR_TRY(check_params(c, p, vol, cams));
    FR_TRY(check_dev(c, out_rgb, image_bytes(cams, ncam), "out_rgb"));
    static thread_local SingleArgs a;
    fill_problem(vol, cams, ncam, p, a);
    a.p.rendered = out_rgb;
    FR_TRY(attach_pairs(c, vol, p, vol->data, a));
    int nt = tiles_of(a.p.W, a.p.H, ncam);
    FR_TRY(order_tiles(c, a, nt));
    FR_CUDA(c, launch_fwd(a, vol->dtype, vol->kind, nt, c->stream));
    return FR_OK;
}

extern "C" fr_status fr_render_residual(fr_ctx* c, const fr_volume* vol, const fr_camera* cams, int ncam,
                                        const fr_params* p, const float* targets, const int32_t* bbox,
                                        float* rendered, float* residual, float* sq_err)
{
    FR_BEGIN(c);
    FR_TRY(check_volume(c, vol, "vol"));
    FR_TRY(check_cams(c, cams, ncam));
    FR_TRY(check_params(c, p, vol, cams));
    const size_t ib = image_bytes(cams, ncam);
    FR_TRY(check_dev(c, targets, ib, "targets"));
    FR_TRY(check_dev(c, bbox, (size_t)ncam * 4 * sizeof(int32_t), "bbox"));
    if (rendered) FR_TRY(check_dev(c, rendered, ib, "rendered"));
    FR_TRY(check_dev(c, residual, ib, "residual"));
    FR_TRY(check_dev(c, sq_err, 4 * sizeof(float), "sq_err"));
    static thread_local SingleArgs a;
    fill_problem(vol, cams, ncam, p, a);
    int nt = tiles_of(a.p.W, a.p.H, ncam);
    FR_TRY(ensure(c, c->partials, (size_t)nt * 4 * sizeof(float), "partials"));
    a.p.targets = targets;
    a.p.bbox = bbox;
    a.p.rendered = rendered;
    a.p.residual = residual;
    a.p.partials = static_cast<float*>(c->partials.p);
    FR_TRY(attach_pairs(c, vol, p, vol->data, a));
    void* fin = nullptr;
    FR_TRY(fin_scratch(c, &fin));
    FR_TRY(order_tiles(c, a, nt));
    FR_CUDA(c, launch_fwd(a, vol->dtype, vol->kind, nt, c->stream));
    FR_CUDA(c, launch_finalize(a.p.partials, nt, sq_err, c->stream, 0, fin));
    return FR_OK;
}

extern "C" fr_status fr_adjust(fr_ctx* c, const fr_volume* vol, const fr_camera* cams, int ncam,
                               const fr_params* p, const float* residual, int iteration, float* dV)
{
    FR_BEGIN(c);
    FR_TRY(check_volume(c, vol, "vol"));
    if (vol->kind != FR_KIND_RGB) return fail(c, FR_EINVAL, "fr_adjust needs an RGB volume (for sigma)");
    FR_TRY(check_cams(c, cams, ncam));
    FR_TRY(check_params(c, p, vol, cams));
    if (iteration < 0 || iteration >= (1 << 20)) return fail(c, FR_EINVAL, "iteration must be in [0, 2^20)");
    FR_TRY(check_dev(c, residual, image_bytes(cams, ncam), "residual"));
    FR_TRY(check_align(c, dV, 16, "dV"));
    FR_TRY(check_dev(c, dV, (size_t)node_count(vol) * 16, "dV"));
    static thread_local SingleArgs a;
    fill_problem(vol, cams, ncam, p, a);
    a.p.img_in = residual;
    a.p.dV = dV;
    a.p.iteration = iteration;
    FR_CUDA(c, launch_adjust(a, vol->dtype, tiles_of(a.p.W, a.p.H, ncam), c->stream));
    return FR_OK;
}

extern "C" fr_status fr_apply_update(fr_ctx* c, fr_volume* vol, float* dV, float scale, int with_sigma,
                                     int clamp_nonneg, int zero_dV)
{
    FR_BEGIN(c);
    FR_TRY(check_volume(c, vol, "vol"));
    if (!std::isfinite(scale)) return fail(c, FR_EINVAL, "scale must be finite");
    const size_t comp = (size_t)rec_components(vol->kind);
    FR_TRY(check_align(c, dV, comp * 4, "dV"));
    FR_TRY(check_dev(c, dV, (size_t)node_count(vol) * comp * 4, "dV"));
    FR_CUDA(c, launch_apply(vol->data, vol->dtype, vol->kind, node_count(vol), dV, scale, with_sigma,
                            clamp_nonneg, zero_dV, c->stream));
    return FR_OK;
}

extern "C" fr_status fr_render_backward(fr_ctx* c, const fr_volume* vol, const fr_camera* cams, int ncam,
                                        const fr_params* p, const float* L_total, const float* grad_img,
                                        float* grad)
{
    FR_BEGIN(c);
    FR_TRY(check_volume(c, vol, "vol"));
    FR_TRY(check_cams(c, cams, ncam));
    FR_TRY(check_params(c, p, vol, cams));
    const size_t ib = image_bytes(cams, ncam);
    FR_TRY(check_dev(c, L_total, ib, "L_total"));
    FR_TRY(check_dev(c, grad_img, ib, "grad_img"));
    const size_t comp = (size_t)rec_components(vol->kind);
    FR_TRY(check_align(c, grad, comp * 4, "grad"));
    FR_TRY(check_dev(c, grad, (size_t)node_count(vol) * comp * 4, "grad"));
    static thread_local SingleArgs a;
    fill_problem(vol, cams, ncam, p, a);
    a.p.img_in = grad_img;
    a.p.L_total = L_total;
    a.p.dV = grad;
    const int nt = tiles_of(a.p.W, a.p.H, ncam);
    FR_TRY(order_tiles(c, a, nt));
    FR_CUDA(c, launch_backward(a, vol->dtype, vol->kind, nt, c->stream));
    return FR_OK;
}

extern "C" fr_status fr_scatter_source(fr_ctx* c, const fr_volume* em, const float* albedo, float* J,
                                       fr_volume* out)
{
    FR_BEGIN(c);
    FR_TRY(check_volume(c, em, "emission"));
    FR_TRY(check_volume(c, out, "out"));
    if (em->kind != FR_KIND_RGB || out->kind != FR_KIND_RGB)
        return fail(c, FR_EINVAL, "in-scattering needs RGB volumes");
    if (em->nx != out->nx || em->ny != out->ny || em->nz != out->nz || em->dtype != out->dtype)
        return fail(c, FR_EINVAL, "emission and out must share grid and storage type");
    if (em->data == out->data) return fail(c, FR_EINVAL, "out must not alias emission");
    const long long n = node_count(em);
    FR_TRY(check_dev(c, albedo, (size_t)n * 4, "albedo"));
    FR_TRY(check_align(c, J, 16, "J"));
    FR_TRY(check_dev(c, J, (size_t)n * 16, "J"));
    FR_CUDA(c, launch_scatter_source(em->data, em->dtype, albedo, J, out->data, out->dtype, em->nx, em->ny,
                                     em->nz, c->stream));
    return FR_OK;
}

extern "C" fr_status fr_planck_lut(fr_ctx* c, float t_min, float t_max, int m, float* lut)
{
    FR_BEGIN(c);
    if (!(t_min > 0.0f) || !(t_max > t_min) || !std::isfinite(t_max) || m < 2 || m > (1 << 20))
        return fail(c, FR_EINVAL, "need 0 < t_min < t_max and 2 <= m <= 2^20");
    FR_TRY(check_align(c, lut, 16, "lut"));
    FR_TRY(check_dev(c, lut, (size_t)m * 16, "lut"));
    FR_CUDA(c, launch_planck_lut(t_min, t_max, m, lut, c->stream));
    return FR_OK;
}

// ---------------------------------------------------------------------------
// Volumes owned by the library
// ---------------------------------------------------------------------------

extern "C" fr_status fr_volume_create(fr_ctx* c, int nx, int ny, int nz, const float origin[3], float h, int kind,
                                      int dtype, fr_volume* out)
{
    FR_BEGIN(c);
    if (!out || !origin) return fail(c, FR_EINVAL, "out and origin must not be NULL");
    fr_volume v{};
    v.nx = nx; v.ny = ny; v.nz = nz;
    v.kind = kind;
    v.dtype = dtype;
    for (int a = 0; a < 3; ++a) v.origin[a] = origin[a];
    v.h = h;
    if (nx < 2 || ny < 2 || nz < 2 || nx > 8192 || ny > 8192 || nz > 8192)
        return fail(c, FR_EINVAL, "extents must be in [2, 8192], got %d x %d x %d", nx, ny, nz);
    if (node_count(&v) >= (1LL << 31)) return fail(c, FR_EINVAL, "at most 2^31 - 1 nodes");
    if (kind != FR_KIND_RGB && kind != FR_KIND_TEMP) return fail(c, FR_EINVAL, "bad kind %d", kind);
    if (dtype != FR_F32 && dtype != FR_BF16 && dtype != FR_F16) return fail(c, FR_EINVAL, "bad dtype %d", dtype);
    if (!(h > 0.0f) || !std::isfinite(h) || !finite3(origin))
        return fail(c, FR_EINVAL, "spacing must be positive and origin finite");
    const size_t bytes = (size_t)node_count(&v) * rec_bytes(&v);
    void* data = nullptr;
    if (cudaMalloc(&data, bytes) != cudaSuccess) {
        cudaGetLastError();
        return fail(c, FR_ENOMEM, "cannot allocate %zu bytes of volume records", bytes);
    }
    cudaError_t e = cudaMemsetAsync(data, 0, bytes, c->stream);
    if (e != cudaSuccess) {
        cudaFree(data);
        return cuda_fail(c, e, "cudaMemsetAsync");
    }
    c->owned.push_back(data);
    v.data = data;
    *out = v;
    return FR_OK;
}

extern "C" fr_status fr_volume_free(fr_ctx* c, fr_volume* vol)
{
    FR_BEGIN(c);
    if (!vol) return fail(c, FR_EINVAL, "vol is NULL");
    auto it = std::find(c->owned.begin(), c->owned.end(), vol->data);
    if (!vol->data || it == c->owned.end())
        return fail(c, FR_EINVAL, "vol was not created by fr_volume_create on this context");
    FR_CUDA(c, cudaStreamSynchronize(c->stream));
    c->owned.erase(it);
    FR_CUDA(c, cudaFree(vol->data));
    vol->data = nullptr;
    return FR_OK;
}

// float32 values of a volume's records (nodes x components)
static size_t volume_values(const fr_volume* v) { return (size_t)node_count(v) * rec_components(v->kind); }

extern "C" fr_status fr_volume_upload(fr_ctx* c, fr_volume* vol, const float* src, int src_is_host)
{
    FR_BEGIN(c);
    FR_TRY(check_volume(c, vol, "vol"));
    if (!src) return fail(c, FR_EINVAL, "src is NULL");
    const size_t n = volume_values(vol), bytes = n * sizeof(float);
    if (!src_is_host) {
        FR_TRY(check_align(c, src, 16, "src"));
        FR_TRY(check_dev(c, src, bytes, "src"));
    }
    const cudaMemcpyKind kind = src_is_host ? cudaMemcpyHostToDevice : cudaMemcpyDeviceToDevice;
    if (vol->dtype == FR_F32) {
        FR_CUDA(c, cudaMemcpyAsync(vol->data, src, bytes, kind, c->stream));
        return FR_OK;
    }
    FR_TRY(check_align(c, vol->data, 8, "vol"));
    const float* d = src;
    if (src_is_host) {
        FR_TRY(ensure(c, c->vol_stage, bytes, "volume staging"));
        FR_CUDA(c, cudaMemcpyAsync(c->vol_stage.p, src, bytes, kind, c->stream));
        d = static_cast<const float*>(c->vol_stage.p);
    }
    FR_CUDA(c, launch_to_storage(d, vol->data, vol->dtype, (long long)n, c->stream));
    return FR_OK;
}

extern "C" fr_status fr_volume_download(fr_ctx* c, const fr_volume* vol, float* dst, int dst_is_host)
{
    FR_BEGIN(c);
    FR_TRY(check_volume(c, vol, "vol"));
    if (!dst) return fail(c, FR_EINVAL, "dst is NULL");
    const size_t n = volume_values(vol), bytes = n * sizeof(float);
    if (!dst_is_host) {
        FR_TRY(check_align(c, dst, 16, "dst"));
        FR_TRY(check_dev(c, dst, bytes, "dst"));
    }
    const cudaMemcpyKind kind = dst_is_host ? cudaMemcpyDeviceToHost : cudaMemcpyDeviceToDevice;
    if (vol->dtype == FR_F32) {
        FR_CUDA(c, cudaMemcpyAsync(dst, vol->data, bytes, kind, c->stream));
    } else {
        FR_TRY(check_align(c, vol->data, 8, "vol"));
        float* d = dst;
        if (dst_is_host) {
            FR_TRY(ensure(c, c->vol_stage, bytes, "volume staging"));
            d = static_cast<float*>(c->vol_stage.p);
        }
        FR_CUDA(c, launch_from_storage(vol->data, d, vol->dtype, (long long)n, c->stream));
        if (dst_is_host) FR_CUDA(c, cudaMemcpyAsync(dst, d, bytes, kind, c->stream));
    }
    if (dst_is_host) FR_CUDA(c, cudaStreamSynchronize(c->stream));
    return FR_OK;
}

// ---------------------------------------------------------------------------
// Camera sets (host memory owned by the library)
// ---------------------------------------------------------------------------

struct fr_cams {
    std::vector<fr_camera> cams;
};

static fr_status cams_finish(std::vector<fr_camera>& v, fr_cams** out)
{
    fr_ctx probe;   // validation messages are not kept: a host-only call has no context
    if (check_cams(&probe, v.data(), (int)v.size()) != FR_OK) return FR_EINVAL;
    fr_cams* c = new (std::nothrow) fr_cams();
    if (!c) return FR_ENOMEM;
    c->cams.swap(v);
    *out = c;
    return FR_OK;
}

extern "C" fr_status fr_cams_create(int k, const double* P, const int32_t* wh, fr_cams** out)
{
    if (!out) return FR_EINVAL;
    *out = nullptr;
    if (k < 1 || k > FR_MAX_VIEWS || !P || !wh) return FR_EINVAL;
    std::vector<fr_camera> v((size_t)k);
    for (int i = 0; i < k; ++i) {
        const fr_status s = fr_camera_from_projection(P + 12 * i, wh[2 * i], wh[2 * i + 1], &v[(size_t)i]);
        if (s != FR_OK) return s;
    }
    return cams_finish(v, out);
}

extern "C" fr_status fr_cams_ring(int k, int width, int height, const float center[3], float radius, float fov_deg,
                                  const float* elevation_deg, float phase, fr_cams** out)
{
    if (!out) return FR_EINVAL;
    *out = nullptr;
    if (k < 1 || k > FR_MAX_VIEWS || !center || !finite3(center) || !(radius > 0.0f) || !std::isfinite(radius) ||
        !(fov_deg > 0.0f && fov_deg < 180.0f) || !std::isfinite(phase))
        return FR_EINVAL;
    const double pi = 3.14159265358979323846;
    std::vector<fr_camera> v((size_t)k);
    for (int i = 0; i < k; ++i) {
        const double th = phase + 2.0 * pi * i / k;
        const double el = elevation_deg ? elevation_deg[i] * pi / 180.0 : 0.0;
        if (!std::isfinite(el) || std::fabs(el) >= 0.5 * pi) return FR_EINVAL;
        const double off[3] = {std::cos(el) * std::cos(th), std::sin(el), std::cos(el) * std::sin(th)};
        // looking at the centre, right = fwd x world up (+y), up = right x fwd
        const double f[3] = {-off[0], -off[1], -off[2]};
        double r[3] = {-f[2], 0.0, f[0]};
        const double rn = std::sqrt(r[0] * r[0] + r[2] * r[2]);
        for (double& x : r) x /= rn;
        const double u[3] = {r[1] * f[2] - r[2] * f[1], r[2] * f[0] - r[0] * f[2], r[0] * f[1] - r[1] * f[0]};
        fr_camera& c = v[(size_t)i];
        memset(&c, 0, sizeof c);
        for (int a = 0; a < 3; ++a) {
            c.pos[a] = (float)(center[a] + radius * off[a]);
            c.right[a] = (float)r[a];
            c.up[a] = (float)u[a];
            c.fwd[a] = (float)f[a];
        }
        c.tan_half_fov = (float)std::tan(0.5 * fov_deg * pi / 180.0);
        c.width = width;
        c.height = height;
    }
    return cams_finish(v, out);
}

extern "C" int32_t fr_cams_count(const fr_cams* c) { return c ? (int32_t)c->cams.size() : 0; }

extern "C" const fr_camera* fr_cams_data(const fr_cams* c) { return c ? c->cams.data() : nullptr; }

extern "C" fr_status fr_cams_destroy(fr_cams* c)
{
    if (!c) return FR_EINVAL;
    delete c;
    return FR_OK;
}

// ---------------------------------------------------------------------------
// Cameras and grids (host arithmetic)
// ---------------------------------------------------------------------------

extern "C" fr_status fr_camera_from_projection(const double P[12], int width, int height, fr_camera* out)
{
    if (!P || !out || width < 1 || height < 1) return FR_EINVAL;
    // RQ decomposition of M = P[:, :3] = K R by Givens rotations: zero M[2][1],
    // then M[2][0], then M[1][0] with rotations about x, y, z applied on the right.
    // P and -P are the same camera: take the sign that gives det(M) > 0, so
    // that R is a proper rotation
    double Pm[12];
    for (int i = 0; i < 12; ++i) Pm[i] = P[i];
    const double detM = Pm[0] * (Pm[5] * Pm[10] - Pm[6] * Pm[9]) - Pm[1] * (Pm[4] * Pm[10] - Pm[6] * Pm[8]) +
                        Pm[2] * (Pm[4] * Pm[9] - Pm[5] * Pm[8]);
    if (!(detM != 0.0) || !std::isfinite(detM)) return FR_EINVAL;
    if (detM < 0.0)
        for (int i = 0; i < 12; ++i) Pm[i] = -Pm[i];
    double M[3][3], Q[3][3] = {{1, 0, 0}, {0, 1, 0}, {0, 0, 1}};
    for (int r = 0; r < 3; ++r)
        for (int c = 0; c < 3; ++c) M[r][c] = Pm[4 * r + c];
    auto rotate = [&](int a, int b, double cth, double sth) {
        // M <- M G, Q <- G^T Q with G the rotation in the (a, b) plane
        for (int r = 0; r < 3; ++r) {
            const double ma = M[r][a], mb = M[r][b];
            M[r][a] = ma * cth + mb * sth;
            M[r][b] = -ma * sth + mb * cth;
        }
        for (int c = 0; c < 3; ++c) {
            const double qa = Q[a][c], qb = Q[b][c];
            Q[a][c] = cth * qa + sth * qb;
            Q[b][c] = -sth * qa + cth * qb;
        }
    };
    auto zero = [&](int row, int a, int b) {   // zero M[row][a] using column b
        const double x = M[row][a], y = M[row][b], r = std::hypot(x, y);
        if (r == 0.0) return;
        rotate(a, b, y / r, -x / r);
    };
    zero(2, 1, 2);
    zero(2, 0, 2);
    zero(1, 0, 1);
    // make K's diagonal positive: flip signs of K's columns and R's rows
    for (int d = 0; d < 3; ++d)
        if (M[d][d] < 0.0) {
            for (int r = 0; r < 3; ++r) M[r][d] = -M[r][d];
            for (int c = 0; c < 3; ++c) Q[d][c] = -Q[d][c];
        }
    if (!(M[2][2] > 0.0)) return FR_EINVAL;
    double K[3][3];
    for (int r = 0; r < 3; ++r)
        for (int c = 0; c < 3; ++c) K[r][c] = M[r][c] / M[2][2];
    const double f = K[0][0], fv = K[1][1], sk = K[0][1], cu = K[0][2], cv = K[1][2];
    if (!(f > 0.0) || std::fabs(sk) > 1e-6 * f || std::fabs(f - fv) > 1e-6 * f) return FR_EINVAL;
    if (std::fabs(cu - 0.5 * (width - 1)) > 1e-3 || std::fabs(cv - 0.5 * (height - 1)) > 1e-3) return FR_EINVAL;
    // centre: the left block is now K' R with K' = M (upper triangular, K
    // scaled by M[2][2]), and p4 = -K' R C, so C = -R^T K'^-1 p4 (back substitution)
    const double p4[3] = {Pm[3], Pm[7], Pm[11]};
    double y[3];
    y[2] = p4[2] / M[2][2];
    y[1] = (p4[1] - M[1][2] * y[2]) / M[1][1];
    y[0] = (p4[0] - M[0][1] * y[1] - M[0][2] * y[2]) / M[0][0];
    fr_camera cam;
    memset(&cam, 0, sizeof cam);
    for (int a = 0; a < 3; ++a) {
        cam.pos[a] = (float)(-(Q[0][a] * y[0] + Q[1][a] * y[1] + Q[2][a] * y[2]));
        cam.right[a] = (float)Q[0][a];
        cam.up[a] = (float)(-Q[1][a]);
        cam.fwd[a] = (float)Q[2][a];
    }
    cam.tan_half_fov = (float)(height / (2.0 * fv));
    cam.width = width;
    cam.height = height;
    *out = cam;
    return FR_OK;
}

extern "C" fr_status fr_volume_dims(const fr_camera* cams, int ncam, const float box_min[3], const float box_max[3],
                                    float alpha, int32_t dims[3], float* h, float n[3])
{
    if (!cams || ncam < 1 || !box_min || !box_max || !dims || !h || !(alpha > 0.0f)) return FR_EINVAL;
    double lo[3], len[3];
    for (int d = 0; d < 3; ++d) {
        lo[d] = box_min[d];
        len[d] = (double)box_max[d] - box_min[d];
        if (!(len[d] > 0.0)) return FR_EINVAL;
    }
    double nmax[3] = {0.0, 0.0, 0.0};
    for (int v = 0; v < ncam; ++v) {
        const fr_camera& c = cams[v];
        const double ty = c.tan_half_fov, tx = ty * c.width / c.height;
        double uv[8][2];
        for (int b = 0; b < 8; ++b) {
            double X[3], xc = 0.0, yc = 0.0, zc = 0.0;
            for (int d = 0; d < 3; ++d) {
                X[d] = (((b >> d) & 1) ? lo[d] + len[d] : lo[d]) - c.pos[d];
                xc += X[d] * c.right[d];
                yc += X[d] * c.up[d];
                zc += X[d] * c.fwd[d];
            }
            if (!(zc > 0.0)) return FR_EINVAL;
            uv[b][0] = (xc / zc / tx + 1.0) * 0.5 * c.width - 0.5;
            uv[b][1] = (1.0 - yc / zc / ty) * 0.5 * c.height - 0.5;
        }
        for (int b = 0; b < 8; ++b)
            for (int d = 0; d < 3; ++d) {
                if ((b >> d) & 1) continue;   // edge from corner b to b + (1 << d), along axis d
                const int e = b | (1 << d);
                const double du = std::fabs(uv[e][0] - uv[b][0]), dv = std::fabs(uv[e][1] - uv[b][1]);
                nmax[d] = std::max(nmax[d], std::max(du, dv));
            }
    }
    double hh = INFINITY;
    for (int d = 0; d < 3; ++d) {
        if (!(nmax[d] > 0.0)) return FR_EINVAL;
        hh = std::min(hh, alpha * len[d] / nmax[d]);
    }
    for (int d = 0; d < 3; ++d) {
        const double cells = std::ceil(len[d] / hh - 1e-9);
        if (cells + 1 > (double)INT_MAX) return FR_EINVAL;
        dims[d] = (int32_t)cells + 1;
        if (n) n[d] = (float)nmax[d];
    }
    *h = (float)hh;
    return FR_OK;
}

extern "C" fr_status fr_temperature_from_green(fr_ctx* c, const fr_volume* rgb, const fr_params* p,
                                               fr_volume* temp)
{
    FR_BEGIN(c);
    if (!p) return fail(c, FR_EINVAL, "p is NULL");
    FR_TRY(check_volume(c, rgb, "rgb"));
    FR_TRY(check_volume(c, temp, "temp"));
    if (rgb->kind != FR_KIND_RGB || temp->kind != FR_KIND_TEMP)
        return fail(c, FR_EINVAL, "rgb must hold RGB records and temp temperature records");
    if (rgb->nx != temp->nx || rgb->ny != temp->ny || rgb->nz != temp->nz)
        return fail(c, FR_EINVAL, "the grids differ");
    if (!p->lut || p->lut_size < 2 || !(p->lut_t_max > p->lut_t_min))
        return fail(c, FR_EINVAL, "needs lut, lut_size >= 2 and lut_t_max > lut_t_min");
    FR_TRY(check_align(c, p->lut, 16, "lut"));
    FR_TRY(check_dev(c, p->lut, (size_t)p->lut_size * 16, "lut"));
    FR_CUDA(c, launch_green_to_temp(rgb->data, rgb->dtype, temp->data, temp->dtype, node_count(rgb), p->lut,
                                    p->lut_size, p->lut_t_min, p->lut_t_max, c->stream));
    return FR_OK;
}

extern "C" fr_status fr_volume_rmse(fr_ctx* c, const fr_volume* a, const fr_volume* b, const uint32_t* tags,
                                    uint32_t full_mask, float* rmse3, int64_t* count)
{
    FR_BEGIN(c);
    if (!rmse3) return fail(c, FR_EINVAL, "rmse3 is NULL");
    FR_TRY(check_volume(c, a, "a"));
    FR_TRY(check_volume(c, b, "b"));
    if (a->kind != FR_KIND_RGB || b->kind != FR_KIND_RGB) return fail(c, FR_EINVAL, "RGB volumes are compared");
    if (a->nx != b->nx || a->ny != b->ny || a->nz != b->nz) return fail(c, FR_EINVAL, "the grids differ");
    const long long nodes = node_count(a);
    if (tags) FR_TRY(check_dev(c, tags, (size_t)nodes * 4, "tags"));
    const int g = volume_err_blocks(nodes);
    FR_TRY(ensure(c, c->verr, align256((size_t)g * 16) + 32, "volume error"));
    float* out = reinterpret_cast<float*>(static_cast<char*>(c->verr.p) + align256((size_t)g * 16));
    FR_CUDA(c, launch_volume_err(a->data, a->dtype, b->data, b->dtype, nodes, tags, full_mask, c->verr.p, out,
                                 c->stream));
    FR_CUDA(c, cudaMemcpyAsync(c->host_counter, out, 24, cudaMemcpyDeviceToHost, c->stream));
    FR_CUDA(c, cudaStreamSynchronize(c->stream));
    const char* hs = reinterpret_cast<const char*>(c->host_counter);
    unsigned long long n = 0;
    memcpy(rmse3, hs, 12);
    memcpy(&n, hs + 16, 8);
    if (count) *count = (int64_t)n;
    return FR_OK;
}

extern "C" fr_status fr_trace_phases(fr_ctx* c, int on)
{
    FR_BEGIN(c);
    c->trace_on = on != 0;
    c->trace_overflow = false;
    c->trace_phase.clear();
    return FR_OK;
}

extern "C" fr_status fr_phase_times(fr_ctx* c, float* ms, int n, int32_t* calls)
{
    FR_BEGIN(c);
    if (!ms || n < FR_PHASE_COUNT) return fail(c, FR_EINVAL, "ms must hold %d entries", (int)FR_PHASE_COUNT);
    for (int i = 0; i < FR_PHASE_COUNT; ++i) ms[i] = 0.0f;
    int32_t nc = 0;
    const size_t ne = c->trace_phase.size();
    if (ne) FR_CUDA(c, cudaEventSynchronize(c->trace_pool[ne - 1]));
    for (size_t i = 0; i < ne; ++i) {
        const int ph = c->trace_phase[i];
        if (ph < 0) {
            ++nc;
            continue;
        }
        if (i == 0) continue;
        float t = 0.0f;
        FR_CUDA(c, cudaEventElapsedTime(&t, c->trace_pool[i - 1], c->trace_pool[i]));
        ms[ph] += t;
    }
    if (calls) *calls = nc;
    const bool over = c->trace_overflow;
    c->trace_phase.clear();
    c->trace_overflow = false;
    if (over) return fail(c, FR_ERANGE, "more than %zu trace events went unread", kTraceMaxEvents);
    return FR_OK;
}

extern "C" fr_status fr_table_stats(const fr_ctx* c, uint64_t stats[4])
{
    if (!c || !stats) return FR_EINVAL;
    for (int i = 0; i < 4; ++i) stats[i] = c->tab_stats[i];
    return FR_OK;
}

extern "C" fr_status fr_count_samples(fr_ctx* c, const fr_volume* vol, const fr_camera* cams, int ncam,
                                      const fr_params* p, const float* residual, int64_t* samples)
{
    FR_BEGIN(c);
    if (!samples) return fail(c, FR_EINVAL, "samples is NULL");
    FR_TRY(check_volume(c, vol, "vol"));
    FR_TRY(check_cams(c, cams, ncam));
    FR_TRY(check_params(c, p, vol, cams));
    if (residual) FR_TRY(check_dev(c, residual, image_bytes(cams, ncam), "residual"));
    FR_TRY(ensure(c, c->counter, sizeof(unsigned long long), "counter"));
    static thread_local SingleArgs a;
    fill_problem(vol, cams, ncam, p, a);
    a.p.img_in = residual;
    a.p.counter = static_cast<unsigned long long*>(c->counter.p);
    // forward samples: those the march evaluates, empty bricks skipped
    if (!residual && skips_empty(vol, p)) FR_TRY(attach_pairs(c, vol, p, vol->data, a));
    // adjustment samples inside fr_reconstruct with given hull tags: bricks
    // without a key point inside the hull are skipped
    if (residual && p->skip_empty && p->use_hull && p->hull_tags && p->rule == FR_RULE_PAPER &&
        !(p->tau > 0.0f)) {
        const int nbx = bricks_along(vol->nx), nby = bricks_along(vol->ny), nbz = bricks_along(vol->nz);
        FR_TRY(check_dev(c, p->hull_tags, (size_t)node_count(vol) * 4, "hull_tags"));
        FR_TRY(ensure(c, c->hull_bricks, brick_table_bytes(vol->nx, vol->ny, vol->nz), "hull bricks"));
        const unsigned full = ncam >= 32 ? 0xffffffffu : ((1u << ncam) - 1u);
        unsigned char* hb = static_cast<unsigned char*>(c->hull_bricks.p);
        FR_CUDA(c, launch_hull_clear(nullptr, vol->dtype, vol->nx, vol->ny, vol->nz, p->hull_tags, full, hb,
                                     c->stream));
        a.p.occ = hb;
        a.p.nbx = nbx;
        a.p.nby = nby;
        a.p.nbz = nbz;
    }
    FR_CUDA(c, cudaMemsetAsync(a.p.counter, 0, sizeof(unsigned long long), c->stream));
    FR_CUDA(c, launch_count(a, tiles_of(a.p.W, a.p.H, ncam), c->stream));
    FR_CUDA(c, cudaMemcpyAsync(c->host_counter, a.p.counter, sizeof(unsigned long long), cudaMemcpyDeviceToHost,
                               c->stream));
    FR_CUDA(c, cudaStreamSynchronize(c->stream));
    *samples = (int64_t)*c->host_counter;
    return FR_OK;
}

// Hull tags of a problem into `tags` (library scratch for the mask tables; the
// cameras travel as launch parameters).
fr_status hull_tags(fr_ctx* c, const SingleArgs& a, const float* targets, float thresh, unsigned* tags)
{
    const ProbDev& P = a.p;
    FR_TRY(ensure(c, c->sat, (size_t)P.ncam * (P.H + 1) * (P.W + 1) * sizeof(unsigned), "flame-mask tables"));
    FR_CUDA(c, launch_visual_hull(a.cams, P.ncam, P.W, P.H, P.nx, P.ny, P.nz, targets, thresh,
                                  static_cast<unsigned*>(c->sat.p), tags, c->stream));
    return FR_OK;
}

extern "C" fr_status fr_visual_hull(fr_ctx* c, const fr_volume* vol, const fr_camera* cams, int ncam,
                                    const float* targets, const fr_params* p, uint32_t* tags)
{
    FR_BEGIN(c);
    FR_TRY(check_volume(c, vol, "vol"));
    FR_TRY(check_cams(c, cams, ncam));
    FR_TRY(check_params(c, p, vol, cams));
    FR_TRY(check_dev(c, targets, image_bytes(cams, ncam), "targets"));
    FR_TRY(check_dev(c, tags, (size_t)node_count(vol) * 4, "tags"));
    static thread_local SingleArgs a;
    fill_problem(vol, cams, ncam, p, a);
    return hull_tags(c, a, targets, p->flame_thresh, reinterpret_cast<unsigned*>(tags));
}

// ---------------------------------------------------------------------------
// The reconstruction loop
// ---------------------------------------------------------------------------

// The loop of fr_reconstruct (stop_delta < 0: exactly `iters` iterations) and
// of fr_reconstruct_until (stop_delta >= 0: at most `iters` iterations, ended
// on the device by the stop criterion inside a conditional CUDA graph).
// The ray weight tables of a problem (tables.cu): the count march, the scans
// (whose totals and per-warp rows the host reads, to size the tables and to
// order the tiles longest first), the fill march.
fr_status build_tables(fr_ctx* c, const SingleArgs& f, const fr_volume* vol, const unsigned* tags, unsigned full,
                       int nt, const TabMemory& mem, TabIter& it, bool& built, size_t* bytes)
{
    built = false;
    if (bytes) *bytes = 0;
    const long long nodes = node_count(vol);
    const long long nw = (long long)nt * (kTileThreads / 32);
    // the hull's key points in Morton order over the smallest cube of 2^m
    // nodes per edge holding the grid, unless that cube has more than 8
    // items per node (then node order)
    KeyOrder order;
    order.nx = vol->nx;
    order.ny = vol->ny;
    order.nz = vol->nz;
    int m = 0;
    while ((1 << m) < std::max(vol->nx, std::max(vol->ny, vol->nz))) ++m;
    order.mbits = m <= 21 && (1LL << (3 * m)) <= 8 * nodes ? m : 0;
    const long long nk = order.count();
    const size_t nb = tab_scan_blocks(std::max(nk, nw));
    size_t at = 0;
    auto carve = [&](size_t n) {
        const size_t o = at;
        at += align256(n);
        return o;
    };
    const size_t o_wrows = carve(nw * 4), o_woff = carve(nw * 4), o_tfl = carve((size_t)nt * 4),
                 o_tfoff = carve((size_t)nt * 4), o_ncnt = carve((size_t)nodes * 4),
                 o_hnode = carve((size_t)nodes * 4), o_hend = carve((size_t)nodes * 4),
                 o_hid = carve((size_t)nodes * 4), o_order = carve((size_t)nt * 4), o_key = carve((size_t)nt * 4),
                 o_bsum = carve(nb * 8), o_tot = carve(4 * 8);
    const size_t scratch_bytes = at;
    char* base = static_cast<char*>(mem.scratch(scratch_bytes));
    if (!base) return mem.status && *mem.status != FR_ENOMEM ? *mem.status : FR_OK;
    TabBuild b{};
    b.tags = tags;
    b.full = full;
    b.wrows = reinterpret_cast<unsigned*>(base + o_wrows);
    b.woff = reinterpret_cast<unsigned*>(base + o_woff);
    b.tfl = reinterpret_cast<unsigned*>(base + o_tfl);
    b.tfoff = reinterpret_cast<unsigned*>(base + o_tfoff);
    b.ncnt = reinterpret_cast<unsigned*>(base + o_ncnt);
    b.hnode = reinterpret_cast<unsigned*>(base + o_hnode);
    b.hid = reinterpret_cast<unsigned*>(base + o_hid);
    b.order = order;
    b.nodes = nodes;
    unsigned* hend = reinterpret_cast<unsigned*>(base + o_hend);
    unsigned long long* totals = reinterpret_cast<unsigned long long*>(base + o_tot);
    static thread_local SingleArgs bf;
    bf = f;
    bf.p.vol = vol->data;
    cudaStream_t s = c->stream;
    FR_CUDA(c, cudaMemsetAsync(b.ncnt, 0, (size_t)nodes * 4, s));
    // the count march's tiles longest first by the samples in the hull's box
    unsigned* order_dev = reinterpret_cast<unsigned*>(base + o_order);
    if (FR_MARCH_ORDER) {
        FR_CUDA(c, launch_tile_order(bf, nt, bf.p.adj_box, reinterpret_cast<unsigned*>(base + o_key), order_dev, s));
        b.torder = order_dev;
    }
    FR_CUDA(c, launch_tab_count(bf, b, vol->dtype, nt, s));
    FR_CUDA(c, launch_tab_scans(b, nt, reinterpret_cast<unsigned long long*>(base + o_bsum), totals, s));
    static_assert(kHostScratchBytes >= 32, "host scratch holds the four totals");
    FR_CUDA(c, cudaMemcpyAsync(c->host_counter, totals, 32, cudaMemcpyDeviceToHost, s));
    // the warps' rows too, for the tile order (pinned: the order's upload
    // below stays asynchronous; a later build writes the buffer only after
    // its own synchronisation, when that upload is done)
    const size_t host_need = (size_t)nw * 4 + (size_t)nt * 4;
    if (c->tab_host_bytes < host_need) {
        FR_CUDA(c, cudaStreamSynchronize(s));
        if (c->tab_host) cudaFreeHost(c->tab_host);
        c->tab_host = nullptr;
        c->tab_host_bytes = 0;
        FR_CUDA(c, cudaMallocHost(&c->tab_host, host_need));
        c->tab_host_bytes = host_need;
    }
    unsigned* wrows_host = static_cast<unsigned*>(c->tab_host);
    unsigned* order_host = wrows_host + nw;
    FR_CUDA(c, cudaMemcpyAsync(wrows_host, b.wrows, (size_t)nw * 4, cudaMemcpyDeviceToHost, s));
    FR_CUDA(c, cudaStreamSynchronize(s));
    unsigned long long tot[4];
    memcpy(tot, c->host_counter, sizeof tot);
    const unsigned long long rows = tot[0], nflame = tot[1], nadj = tot[2], nhull = tot[3];
    if (bytes) *bytes = scratch_bytes;
    if (rows * 32 >= (1ull << 32) || nadj >= (1ull << 32)) return FR_OK;
    // the tables' block: forward entries, adjustment entries, residuals, staged records
    const size_t t_fwd = align256((size_t)rows * 32 * 8), t_adj = align256((size_t)nadj * 8),
                 t_dl = align256((size_t)nflame * 16), t_hs = align256((size_t)nhull * rec_bytes(vol));
    char* tb = static_cast<char*>(mem.tables(t_fwd + t_adj + t_dl + t_hs));
    if (!tb) return mem.status && *mem.status != FR_ENOMEM ? *mem.status : FR_OK;
    if (bytes) *bytes += t_fwd + t_adj + t_dl + t_hs;
    b.efwd = reinterpret_cast<uint2*>(tb);
    b.eadj = reinterpret_cast<uint2*>(tb + t_fwd);
    b.nadj = nadj;
    b.nhull = (unsigned)nhull;
    // the tiles, longest first, for the fill and for every iteration's forward
    tab_tile_order(wrows_host, nt, order_host);
    FR_CUDA(c, cudaMemcpyAsync(order_dev, order_host, (size_t)nt * 4, cudaMemcpyHostToDevice, s));
    b.torder = order_dev;
    FR_CUDA(c, launch_tab_fill(bf, b, vol->dtype, nt, s));
    FR_CUDA(c, launch_tab_hend(b.hnode, b.ncnt, (unsigned)nhull, hend, s));
    FR_CUDA(c, launch_tab_sort(b.eadj, hend, (unsigned)nhull, s));
    it = TabIter{};
    it.torder = order_dev;
    it.wrows = b.wrows;
    it.woff = b.woff;
    it.tfoff = b.tfoff;
    it.efwd = b.efwd;
    it.eadj = b.eadj;
    it.hnode = b.hnode;
    it.hend = hend;
    it.hs = tb + t_fwd + t_adj + t_dl;
    it.dl = reinterpret_cast<float4*>(tb + t_fwd + t_adj);
    it.nhull = (unsigned)nhull;
    it.nflame = (unsigned)nflame;
    it.nadj = (unsigned)nadj;
    c->tab_stats[0] = rows * 32;
    c->tab_stats[1] = nadj;
    c->tab_stats[2] = nflame;
    c->tab_stats[3] = nhull;
    built = true;
    return FR_OK;
}

// build_tables' memory from the context's scratch (held from call to call,
// under the context's scratch limit)
static TabMemory ctx_tab_memory(fr_ctx* c, fr_status* status)
{
    TabMemory m;
    m.status = status;
    m.scratch = [c, status](size_t n) -> void* {
        *status = ensure(c, c->tab_small, n, "table counts");
        if (*status == FR_ENOMEM) c->err[0] = '\0';
        return *status == FR_OK ? c->tab_small.p : nullptr;
    };
    m.tables = [c, status](size_t n) -> void* {
        *status = ensure(c, c->tab_fwd, n, "ray weight tables");
        if (*status == FR_ENOMEM) c->err[0] = '\0';
        return *status == FR_OK ? c->tab_fwd.p : nullptr;
    };
    return m;
}

static fr_status reconstruct_impl(fr_ctx* c, fr_volume* vol, const float* albedo, const fr_camera* cams, int ncam,
                                  const float* targets, int targets_are_host, const int32_t* bbox, int iters,
                                  int first_iteration, const fr_params* p, float* rmse, int rmse_is_host,
                                  float stop_delta, int32_t* iters_done)
{
    FR_BEGIN(c);
    const bool until = stop_delta >= 0.0f;
    FR_TRY(check_volume(c, vol, "vol"));
    FR_TRY(check_cams(c, cams, ncam));
    FR_TRY(check_params(c, p, vol, cams));
    if (iters < 0) return fail(c, FR_EINVAL, "iters must be >= 0");
    if (first_iteration < 0 || (long long)first_iteration + iters > (1 << 20))
        return fail(c, FR_EINVAL, "iterations must stay below 2^20");
    if (p->rule != FR_RULE_PAPER && p->rule != FR_RULE_GRADIENT) return fail(c, FR_EINVAL, "bad rule");
    if (vol->kind == FR_KIND_TEMP && p->rule == FR_RULE_PAPER)
        return fail(c, FR_EINVAL, "temperature volumes are reconstructed with FR_RULE_GRADIENT");
    if (albedo && vol->kind != FR_KIND_RGB) return fail(c, FR_EINVAL, "albedo needs an RGB volume");
    if (p->rule == FR_RULE_GRADIENT && !std::isfinite(p->grad_step))
        return fail(c, FR_EINVAL, "grad_step must be finite");
    if (!(p->hg_g > -1.0f && p->hg_g < 1.0f)) return fail(c, FR_EINVAL, "hg_g must lie in (-1, 1)");
    if (p->sequential_views != 0 && p->sequential_views != 1)
        return fail(c, FR_EINVAL, "sequential_views must be 0 or 1");
    // views rendered and adjusted one at a time: anisotropic scattering (each
    // view its own source) or the sequential order
    const bool per_view = (p->hg_g != 0.0f && albedo) || p->sequential_views;
    const long long nodes = node_count(vol);
    const size_t ib = image_bytes(cams, ncam);
    if (!targets) return fail(c, FR_EINVAL, "targets is NULL");
    if (!targets_are_host) FR_TRY(check_dev(c, targets, ib, "targets"));
    FR_TRY(check_dev(c, bbox, (size_t)ncam * 4 * sizeof(int32_t), "bbox"));
    if (albedo) FR_TRY(check_dev(c, albedo, (size_t)nodes * 4, "albedo"));
    if (rmse && !rmse_is_host) FR_TRY(check_dev(c, rmse, (size_t)iters * 3 * sizeof(float), "rmse"));
    if (iters == 0) return FR_OK;

    const int comp = rec_components(vol->kind);
    const int nt = tiles_of(cams[0].width, cams[0].height, ncam);
    FR_TRY(ensure(c, c->residual, ib, "residual"));
    FR_TRY(ensure(c, c->dV, (size_t)nodes * comp * 4, "dV"));
    FR_TRY(ensure(c, c->partials, (size_t)nt * 16, "partials"));
    FR_TRY(ensure(c, c->sqerr, (size_t)iters * 16, "sqerr"));
    FR_TRY(ensure(c, c->rmse, (size_t)iters * 12, "rmse"));
    if (targets_are_host) FR_TRY(ensure(c, c->targets, ib, "targets"));
    if (p->rule == FR_RULE_GRADIENT) FR_TRY(ensure(c, c->rendered, ib, "rendered"));
    if (albedo) {
        FR_TRY(ensure(c, c->J, (size_t)nodes * 16, "J"));
        FR_TRY(ensure(c, c->src, (size_t)nodes * rec_bytes(vol), "source"));
    }
    const long long npix = (long long)ncam * cams[0].width * cams[0].height;
    if (npix >= (1LL << 32)) return fail(c, FR_EINVAL, "at most 2^32 pixels per reconstruction");
    // Views pipelined (FR_PIPELINE_VIEWS): the forward march of each view on
    // the context's stream, the adjustment of its flame rays on a second
    // stream as soon as that view's forward is done, so that the forward
    // (latency-bound) and the adjustment (issue-bound) of different views share
    // the SMs.  The adjustment of a view depends on that view's forward alone;
    // the update waits for all of them.  Not with phase tracing (whose events
    // time the kernels one after another) nor inside the stop-criterion graph.
    const bool pipe = FR_PIPELINE_VIEWS && !until && !c->trace_on && !per_view && ncam > 1 &&
                      p->rule == FR_RULE_PAPER;
    const int count_slots = per_view || pipe ? ncam : 1;   // flame-ray counts per iteration
    FR_TRY(ensure(c, c->flame_cnt, (size_t)iters * count_slots * sizeof(unsigned), "flame counts"));
    const bool hg = per_view && p->hg_g != 0.0f && albedo;
    if (hg) FR_TRY(ensure(c, c->L6, (size_t)nodes * 6 * 16, "directional radiances"));
    if (until) FR_TRY(ensure(c, c->loop, 16, "loop counter"));
    // Flame-ray list: one entry per flame pixel and part of its ray, each part's
    // block of a tile's run padded to whole warps (at most one tile's worth per
    // tile and part); the part index sits in an entry's top two bits, so larger
    // reconstructions list whole rays.
#if FR_ADJ_SPLIT > 1
    const bool split = p->rule == FR_RULE_PAPER && npix < (1LL << 30) - 1;
    const int parts = split ? FR_ADJ_SPLIT : 1;
#else
    const bool split = false;
    const int parts = 1;
#endif
    FR_TRY(ensure(c, c->flame_list, (size_t)nt * kTileThreads * parts * sizeof(unsigned), "flame list"));
    if (split) FR_TRY(ensure(c, c->flame_tm, (size_t)nt * kTileThreads * parts * sizeof(float), "flame list"));
    // the flame rays' residuals beside their list entries instead of the
    // residual image (the loop over all views at once, paper rule)
    const bool list_dl = FR_LIST_DL && p->rule == FR_RULE_PAPER && !per_view && !pipe;
    if (list_dl) FR_TRY(ensure(c, c->flame_dl, (size_t)nt * kTileThreads * parts * 3 * sizeof(float), "flame list"));
    FR_TRY(ensure(c, c->pairs, (size_t)nodes * 2 * rec_bytes(vol), "pairs"));
    const int nbx = bricks_along(vol->nx), nby = bricks_along(vol->ny), nbz = bricks_along(vol->nz);
    unsigned char* occ = nullptr;
    if (skips_empty(vol, p)) {
        FR_TRY(ensure(c, c->occ, brick_table_bytes(vol->nx, vol->ny, vol->nz), "brick occupancy"));
        occ = static_cast<unsigned char*>(c->occ.p);
    }
    if (p->use_hull) {
        if (vol->kind != FR_KIND_RGB) return fail(c, FR_EINVAL, "the visual hull applies to RGB volumes");
        if (p->hull_tags) FR_TRY(check_dev(c, p->hull_tags, (size_t)nodes * 4, "hull_tags"));
        else FR_TRY(ensure(c, c->hull, (size_t)nodes * 4, "hull"));
        FR_TRY(ensure(c, c->hull_bricks, brick_table_bytes(vol->nx, vol->ny, vol->nz), "hull bricks"));
    }
    cudaStream_t s = c->stream;
    if (pipe) {
        if (!c->aux) FR_CUDA(c, cudaStreamCreateWithFlags(&c->aux, cudaStreamNonBlocking));
        for (int v = 0; v <= kMaxViews; ++v)
            if (!c->pipe_ev[v]) FR_CUDA(c, cudaEventCreateWithFlags(&c->pipe_ev[v], cudaEventDisableTiming));
    }
    const float* tg = targets;
    if (targets_are_host) {
        FR_CUDA(c, cudaMemcpyAsync(c->targets.p, targets, ib, cudaMemcpyHostToDevice, s));
        tg = static_cast<const float*>(c->targets.p);
    }
    const size_t dv_bytes = (size_t)nodes * comp * 4;
    if (c->dV_zero_at != c->dV.p || c->dV_zero_bytes < dv_bytes) FR_CUDA(c, cudaMemsetAsync(c->dV.p, 0, dv_bytes, s));
    c->dV_zero_at = nullptr;   // until this call completes
    auto loop_done = [&]() {
        c->dV_zero_at = c->dV.p;
        c->dV_zero_bytes = dv_bytes;
    };

    static thread_local SingleArgs f, u;
    fill_problem(vol, cams, ncam, p, f);
    const void* render_vol = albedo ? c->src.p : vol->data;
    f.p.vol = render_vol;
    f.p.targets = tg;
    f.p.bbox = bbox;
    f.p.residual = static_cast<float*>(c->residual.p);
    f.p.partials = static_cast<float*>(c->partials.p);
    f.p.rendered = p->rule == FR_RULE_GRADIENT ? static_cast<float*>(c->rendered.p) : nullptr;
    f.p.pairs = c->pairs.p;
    f.p.occ = occ;
    f.p.occ_box = occ ? brick_box(occ, nbx, nby, nbz) : nullptr;
    f.p.nbx = nbx;
    f.p.nby = nby;
    f.p.nbz = nbz;
    u = f;
    u.p.pairs = nullptr;
    u.p.occ = nullptr;
    u.p.occ_box = nullptr;
    u.p.adj_occ = nullptr;
    u.p.targets = nullptr;
    u.p.partials = nullptr;
    u.p.residual = nullptr;
    u.p.rendered = nullptr;
    u.p.img_in = static_cast<const float*>(c->residual.p);
    u.p.dV = static_cast<float*>(c->dV.p);
    float* sq = static_cast<float*>(c->sqerr.p);
    // flame rays: the forward march of iteration `it` lists them, counted at
    // flame_cnt[it], for the adjustment that follows it
    unsigned* flame_cnt = static_cast<unsigned*>(c->flame_cnt.p);
    unsigned* flame_list = static_cast<unsigned*>(c->flame_list.p);
    FR_TRY(trace_mark(c, -1));
    if (p->rule == FR_RULE_PAPER) {
        FR_CUDA(c, cudaMemsetAsync(flame_cnt, 0, (size_t)iters * count_slots * sizeof(unsigned), s));
        f.p.flist = flame_list;
        f.p.flist_tm = split ? static_cast<float*>(c->flame_tm.p) : nullptr;
        if (list_dl) {
            f.p.flist_dl = static_cast<float*>(c->flame_dl.p);
            f.p.residual = nullptr;
            u.p.flist_dl = f.p.flist_dl;
        }
    }
    const float* flame_tm = split ? static_cast<const float*>(c->flame_tm.p) : nullptr;
    const unsigned* hull = nullptr;
    const unsigned full = ncam >= 32 ? 0xffffffffu : ((1u << ncam) - 1u);
    if (p->use_hull) {
        if (p->hull_tags) {
            hull = p->hull_tags;
        } else {
            FR_TRY(hull_tags(c, f, tg, p->flame_thresh, static_cast<unsigned*>(c->hull.p)));
            hull = static_cast<const unsigned*>(c->hull.p);
        }
        unsigned char* hb = nullptr;
        if (p->skip_empty && p->rule == FR_RULE_PAPER && !(p->tau > 0.0f))
            hb = static_cast<unsigned char*>(c->hull_bricks.p);
        FR_CUDA(c, launch_hull_clear(vol->data, vol->dtype, vol->nx, vol->ny, vol->nz, hull, full, hb, s));
        u.p.adj_occ = hb;
        u.p.adj_box = hb ? brick_box(hb, nbx, nby, nbz) : nullptr;
    }
    // With the hull's brick table, records outside its flagged bricks are
    // zero: the pack skips their nodes and the forward clips its rays to the
    // table's box (which holds every brick with a non-zero record), so the
    // box of the non-zero bricks is not recomputed every iteration.
    const unsigned char* pack_keep = occ ? u.p.adj_occ : nullptr;
    if (pack_keep) f.p.occ_box = u.p.adj_box;
    // The same box bounds the in-scattering sweeps and the update: every record
    // outside it is zero (the hull clear) and no adjustment reaches it
    // (FR_NODE_BOX = 0: the whole grid).
    const NodeBox nbox = FR_NODE_BOX && pack_keep ? NodeBox{u.p.adj_box, nbx, nby, nbz} : NodeBox{};
    // the forward clips to the adjustment's box: the half rays divide the
    // samples inside it (FR_SPLIT_BOX = 0: the whole chord)
    if (FR_SPLIT_BOX && pack_keep) {
        f.p.split_box = u.p.split_box = 1;
        f.p.adj_box = u.p.adj_box;
    }
    // With the box, the last in-scattering sweep writes the x-pair records and
    // the brick marks itself (the pair pack folded into it; FR_SWEEP_PACK = 0:
    // a separate pack)
    const bool fold_pack = FR_SWEEP_PACK && albedo && !hg && nbox.box && occ &&
                           sweeps_take_box(vol->nx, vol->ny, vol->nz);
    const PackOut pk = fold_pack ? PackOut{c->pairs.p, occ} : PackOut{};
    const size_t occ_bytes = brick_table_bytes(vol->nx, vol->ny, vol->nz);
    // The ray weight tables in place of the two marches (fr_params.tables):
    // paper rule, RGB records, the hull's brick table (skip_empty, field
    // mode), G(s) = 1 and all views at once.
    TabIter tab{};
    bool tables = false;
    memset(c->tab_stats, 0, sizeof c->tab_stats);
    if (!FR_FUSED && p->tables != 1 && p->rule == FR_RULE_PAPER && vol->kind == FR_KIND_RGB && hull &&
        u.p.adj_occ && !(p->g_std > 0.0f) && !per_view && !pipe &&
        (p->tables == 2 || iters >= FR_TABLES_MIN_ITERS)) {
        static thread_local SingleArgs tb;
        tb = f;
        tb.p.targets = tg;
        tb.p.adj_occ = u.p.adj_occ;
        tb.p.adj_box = u.p.adj_box;
        fr_status ms = FR_OK;
        FR_TRY(build_tables(c, tb, vol, hull, full, nt, ctx_tab_memory(c, &ms), tab, tables));
    }
    // Marching all views at once: the forward takes its tiles longest first
    // (samples inside the hull's box per ray, else the whole chord), so the
    // grid does not end on the longest tiles
    if (!tables && !per_view && !pipe && !FR_FUSED && FR_MARCH_ORDER) {
        FR_TRY(ensure(c, c->torder, (size_t)nt * 8, "tile order"));
        unsigned* key = static_cast<unsigned*>(c->torder.p);
        FR_CUDA(c, launch_tile_order(f, nt, pack_keep ? u.p.adj_box : nullptr, key, key + nt, s));
        f.p.tile_order = key + nt;
    }
    void* fin = nullptr;
    FR_TRY(fin_scratch(c, &fin));
    float* rmse_dev = static_cast<float*>(c->rmse.p);
    FR_TRY(trace_mark(c, FR_PHASE_SETUP));
    // One iteration on stream st.  it >= 0: per-iteration slots it; it < 0:
    // slot 0 and the iteration index read on the device (graph body).
    // Per-view problems: view v of the call as a one-view problem over the
    // same volume, its targets, box, residual and image slices, its own flame
    // count, and its index v in the G(s) stream.
    const size_t view_px = (size_t)cams[0].width * cams[0].height;
    const int nt1 = tiles_of(cams[0].width, cams[0].height, 1);
    static thread_local SingleArgs fv, uv;
    auto view_problem = [&](int v, int slot) {
        fv = f;
        fv.p.ncam = 1;
        fv.cams[0] = f.cams[v];
        fv.p.targets = tg + 3 * view_px * v;
        fv.p.bbox = bbox + 4 * v;
        fv.p.residual = f.p.residual + 3 * view_px * v;
        if (f.p.rendered) fv.p.rendered = f.p.rendered + 3 * view_px * v;
        fv.p.flist_count = f.p.flist ? flame_cnt + (size_t)slot * count_slots + v : nullptr;
        uv = u;
        uv.p.ncam = 1;
        uv.cams[0] = u.cams[v];
        uv.p.img_in = u.p.img_in + 3 * view_px * v;
        if (p->rule == FR_RULE_GRADIENT) uv.p.L_total = static_cast<const float*>(c->rendered.p) + 3 * view_px * v;
        uv.p.view_base = v;
    };
    // Henyey-Greenstein weights towards each camera (Eq. 9): light travelling
    // along axis direction d comes from -e_d, weight ~ p(omega, -e_d),
    // normalised to sum to 1; omega from the volume's centre to the camera.
    auto hg_weights = [&](int v) {
        HgWeights w;
        const double g = p->hg_g;
        double om[3], len = 0.0;
        const int n[3] = {vol->nx, vol->ny, vol->nz};
        for (int a = 0; a < 3; ++a) {
            om[a] = (double)cams[v].pos[a] - ((double)vol->origin[a] + 0.5 * (n[a] - 1) * (double)vol->h);
            len += om[a] * om[a];
        }
        len = std::sqrt(len);
        double pw[6], sum = 0.0;
        for (int d = 0; d < 6; ++d) {
            const double e = (d & 1) ? -1.0 : 1.0;
            const double cos_wi = -e * om[d / 2] / len;
            const double den = 1.0 + g * g + 2.0 * g * cos_wi;
            pw[d] = (1.0 - g * g) / (den * std::sqrt(den));   // the 1/(4 pi) cancels
            sum += pw[d];
        }
        for (int d = 0; d < 6; ++d) w.w[d] = (float)(pw[d] / sum);
        return w;
    };
    auto per_view_iteration = [&](cudaStream_t st, int it) -> fr_status {
        const int slot = it < 0 ? 0 : it;
        const bool seq = p->sequential_views != 0;
        for (int v = 0; v < ncam; ++v) {
            if (albedo) {
                if (hg) {
                    if (v == 0 || seq)
                        FR_CUDA(c, launch_scatter_L6(vol->data, vol->dtype, static_cast<float*>(c->L6.p), vol->nx,
                                                     vol->ny, vol->nz, st, p->skip_empty != 0));
                    FR_CUDA(c, launch_source_hg(vol->data, vol->dtype, albedo, static_cast<const float*>(c->L6.p),
                                                hg_weights(v), c->src.p, nodes, st));
                } else if (v == 0 || seq) {
                    if (fold_pack) FR_CUDA(c, cudaMemsetAsync(occ, 0, occ_bytes, st));
                    FR_CUDA(c, launch_scatter_source(vol->data, vol->dtype, albedo, static_cast<float*>(c->J.p),
                                                     c->src.p, vol->dtype, vol->nx, vol->ny, vol->nz, st,
                                                     p->skip_empty != 0, nbox, pk));
                }
                FR_TRY(trace_mark(c, FR_PHASE_SCATTER));
            }
            if ((v == 0 || seq || hg) && !fold_pack) {
                FR_CUDA(c, launch_pair_pack(render_vol, c->pairs.p, vol->dtype, vol->kind, vol->nx, vol->ny, vol->nz,
                                            occ, st, pack_keep, nbox));
                FR_TRY(trace_mark(c, FR_PHASE_PACK));
            }
            view_problem(v, slot);
            FR_CUDA(c, launch_fwd(fv, vol->dtype, vol->kind, nt1, st));
            FR_TRY(trace_mark(c, FR_PHASE_FORWARD));
            FR_CUDA(c, launch_finalize(fv.p.partials, nt1, sq + 4 * slot, st, v > 0, fin,
                                       it < 0 ? nullptr : rmse_dev + 3 * slot));
            FR_TRY(trace_mark(c, FR_PHASE_REDUCE));
            if (p->rule == FR_RULE_PAPER) {
                uv.p.iteration = first_iteration + slot;
                FR_CUDA(c, launch_adjust_list(uv, vol->dtype, nt1, flame_list, fv.p.flist_count, st, flame_tm));
            } else {
                uv.p.img_scale = -1.0f;
                FR_CUDA(c, launch_backward(uv, vol->dtype, vol->kind, nt1, st));
            }
            FR_TRY(trace_mark(c, FR_PHASE_ADJUST));
            if (seq || v == ncam - 1) {
                // the update, with the hull clear fused in
                if (p->rule == FR_RULE_PAPER)
                    FR_CUDA(c, launch_apply_box(vol->data, vol->dtype, vol->kind, vol->nx, vol->ny, vol->nz, u.p.dV,
                                                1.0f, 0, p->clamp_nonneg, 1, st, hull, full, nbox));
                else
                    FR_CUDA(c, launch_apply(vol->data, vol->dtype, vol->kind, nodes, u.p.dV, -p->grad_step,
                                            p->update_sigma, p->clamp_nonneg, 1, st, hull, full));
                FR_TRY(trace_mark(c, FR_PHASE_APPLY));
            }
        }
        return FR_OK;
    };
    // The forward and adjustment of an iteration view by view, the
    // adjustments on the second stream (see `pipe`); each view's flame rays in
    // their own region of the list, counted at their own slot.
    const size_t view_region = (size_t)nt1 * kTileThreads * parts;
    auto pipelined_views = [&](cudaStream_t st, int slot) -> fr_status {
        for (int v = 0; v < ncam; ++v) {
            view_problem(v, slot);
            fv.p.flist = flame_list + v * view_region;
            fv.p.flist_tm = split ? static_cast<float*>(c->flame_tm.p) + v * view_region : nullptr;
            FR_CUDA(c, launch_fwd(fv, vol->dtype, vol->kind, nt1, st));
            FR_CUDA(c, launch_finalize(fv.p.partials, nt1, sq + 4 * slot, st, v > 0, fin,
                                       v == ncam - 1 ? rmse_dev + 3 * slot : nullptr));
            FR_CUDA(c, cudaEventRecord(c->pipe_ev[v], st));
            FR_CUDA(c, cudaStreamWaitEvent(c->aux, c->pipe_ev[v], 0));
            uv.p.iteration = first_iteration + slot;
            FR_CUDA(c, launch_adjust_list(uv, vol->dtype, nt1, fv.p.flist, fv.p.flist_count, c->aux,
                                          fv.p.flist_tm));
        }
        FR_CUDA(c, cudaEventRecord(c->pipe_ev[kMaxViews], c->aux));
        FR_CUDA(c, cudaStreamWaitEvent(st, c->pipe_ev[kMaxViews], 0));
        return FR_OK;
    };
    auto one_iteration = [&](cudaStream_t st, int it) -> fr_status {
        if (per_view) return per_view_iteration(st, it);
        const int slot = it < 0 ? 0 : it;
        if (tables) {
            // in-scattering source (no x-pairs: the forward table gathers
            // the source records), rendering and residuals from the forward
            // table, error sums, adjustment and update of the hull's key
            // points from the adjustment table
            if (albedo) {
                FR_CUDA(c, launch_scatter_source(vol->data, vol->dtype, albedo, static_cast<float*>(c->J.p),
                                                 c->src.p, vol->dtype, vol->nx, vol->ny, vol->nz, st,
                                                 p->skip_empty != 0, nbox, PackOut{}));
                FR_TRY(trace_mark(c, FR_PHASE_SCATTER));
            }
            FR_CUDA(c, launch_tab_stage(render_vol, vol->dtype, tab, st));
            FR_CUDA(c, launch_tab_forward(f, tab, vol->dtype, nt, st));
            FR_TRY(trace_mark(c, FR_PHASE_FORWARD));
            // the error sums run inside the adjustment's launch
            const FinArgs fa{f.p.partials, nt, sq + 4 * slot, fin, it < 0 ? nullptr : rmse_dev + 3 * slot};
            if (!FR_TAB_FIN_FUSED) {
                FR_CUDA(c, launch_finalize(fa.partials, nt, fa.out4, st, 0, fin, fa.rmse3));
                FR_TRY(trace_mark(c, FR_PHASE_REDUCE));
            }
            FR_CUDA(c, launch_tab_adjust(vol->data, vol->dtype, nodes, tab, p->clamp_nonneg, st,
                                         FR_TAB_FIN_FUSED ? &fa : nullptr));
            FR_TRY(trace_mark(c, FR_PHASE_ADJUST));
            return FR_OK;
        }
        if (albedo) {
            if (fold_pack) FR_CUDA(c, cudaMemsetAsync(occ, 0, occ_bytes, st));
            FR_CUDA(c, launch_scatter_source(vol->data, vol->dtype, albedo, static_cast<float*>(c->J.p), c->src.p,
                                             vol->dtype, vol->nx, vol->ny, vol->nz, st, p->skip_empty != 0, nbox, pk));
            FR_TRY(trace_mark(c, FR_PHASE_SCATTER));
        }
        if (!fold_pack) {
            FR_CUDA(c, launch_pair_pack(render_vol, c->pairs.p, vol->dtype, vol->kind, vol->nx, vol->ny, vol->nz, occ,
                                        st, pack_keep, nbox));
            FR_TRY(trace_mark(c, FR_PHASE_PACK));
        }
        if (pipe) {
            FR_TRY(pipelined_views(st, slot));
            FR_CUDA(c, launch_apply_box(vol->data, vol->dtype, vol->kind, vol->nx, vol->ny, vol->nz, u.p.dV, 1.0f,
                                        0, p->clamp_nonneg, 1, st, hull, full, nbox));
            return FR_OK;
        }
#if FR_FUSED
        if (p->rule == FR_RULE_PAPER && f.p.pairs && occ && !(p->tau > 0.0f) && vol->kind == FR_KIND_RGB) {
            // (comparison build: the forward and the adjustment in one kernel)
            static thread_local SingleArgs fu;
            fu = f;
            fu.p.flist = nullptr;
            fu.p.flist_tm = nullptr;
            fu.p.flist_count = nullptr;
            fu.p.residual = nullptr;
            fu.p.dV = u.p.dV;
            fu.p.adj_occ = u.p.adj_occ;
            fu.p.adj_box = u.p.adj_box;
            fu.p.iteration = first_iteration + slot;
            fu.p.iter_dev = u.p.iter_dev;
            FR_CUDA(c, launch_fused(fu, vol->dtype, nt, st));
            FR_TRY(trace_mark(c, FR_PHASE_FORWARD));
            FR_CUDA(c, launch_finalize(f.p.partials, nt, sq + 4 * slot, st, 0, fin,
                                       it < 0 ? nullptr : rmse_dev + 3 * slot));
            FR_TRY(trace_mark(c, FR_PHASE_REDUCE));
            FR_CUDA(c, launch_apply_box(vol->data, vol->dtype, vol->kind, vol->nx, vol->ny, vol->nz, u.p.dV, 1.0f,
                                        0, p->clamp_nonneg, 1, st, hull, full, nbox));
            FR_TRY(trace_mark(c, FR_PHASE_APPLY));
            return FR_OK;
        }
#endif
        f.p.flist_count = f.p.flist ? flame_cnt + slot : nullptr;
        FR_CUDA(c, launch_fwd(f, vol->dtype, vol->kind, nt, st));
        FR_TRY(trace_mark(c, FR_PHASE_FORWARD));
        // the error sums and (outside the graph loop, whose converge kernel
        // records it) the error measure of this iteration
        FR_CUDA(c, launch_finalize(f.p.partials, nt, sq + 4 * slot, st, 0, fin,
                                   it < 0 ? nullptr : rmse_dev + 3 * slot));
        FR_TRY(trace_mark(c, FR_PHASE_REDUCE));
        if (p->rule == FR_RULE_PAPER) {
            u.p.iteration = first_iteration + slot;
            FR_CUDA(c, launch_adjust_list(u, vol->dtype, nt, flame_list, flame_cnt + slot, st, flame_tm));
            FR_TRY(trace_mark(c, FR_PHASE_ADJUST));
#ifdef FR_ADJ_GATHER_PROBE
            // (measurement build: a gather's set-up work, timed as the finish phase)
            if (hull) {
                FR_TRY(ensure(c, c->probe, (size_t)nodes * 8 + 256, "gather probe"));
                unsigned* pl = static_cast<unsigned*>(c->probe.p);
                FR_CUDA(c, launch_gather_probe(u, hull, full, nodes, pl, pl + 2 * nodes,
                                               reinterpret_cast<float*>(pl + nodes), st));
                FR_TRY(trace_mark(c, FR_PHASE_FINISH));
            }
#endif
            FR_CUDA(c, launch_apply_box(vol->data, vol->dtype, vol->kind, vol->nx, vol->ny, vol->nz, u.p.dV, 1.0f,
                                        0, p->clamp_nonneg, 1, st, hull, full, nbox));
        } else {
            // d(0.5 sum m dL^2)/d(rendered) = -m dL: the residual scaled by -1
            u.p.img_scale = -1.0f;
            u.p.L_total = static_cast<const float*>(c->rendered.p);
            FR_CUDA(c, launch_backward(u, vol->dtype, vol->kind, nt, st));
            FR_TRY(trace_mark(c, FR_PHASE_ADJUST));
            FR_CUDA(c, launch_apply(vol->data, vol->dtype, vol->kind, nodes, u.p.dV, -p->grad_step,
                                    p->update_sigma, p->clamp_nonneg, 1, st, hull, full));
        }
        FR_TRY(trace_mark(c, FR_PHASE_APPLY));
        return FR_OK;
    };
    if (!until) {
        for (int it = 0; it < iters; ++it) FR_TRY(one_iteration(s, it));
        loop_done();
        FR_TRY(trace_mark(c, FR_PHASE_FINISH));
        if (rmse) {
            if (rmse_is_host) {
                FR_CUDA(c, cudaMemcpyAsync(rmse, c->rmse.p, (size_t)iters * 12, cudaMemcpyDeviceToHost, s));
                FR_CUDA(c, cudaStreamSynchronize(s));
            } else {
                FR_CUDA(c, cudaMemcpyAsync(rmse, c->rmse.p, (size_t)iters * 12, cudaMemcpyDeviceToDevice, s));
            }
        }
        return FR_OK;
    }

    // Until the stop criterion: a graph whose conditional while node runs the
    // iteration body; the body's last kernel records the iteration's error,
    // advances the device iteration counter and ends the loop.  Graph bodies
    // hold no event records, so tracing pauses during the capture.
    int* loop_iter = static_cast<int*>(c->loop.p);
    FR_CUDA(c, cudaMemsetAsync(loop_iter, 0, sizeof(int), s));
    u.p.iter_dev = loop_iter;
    if (!c->capture) FR_CUDA(c, cudaStreamCreateWithFlags(&c->capture, cudaStreamNonBlocking));
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    FR_CUDA(c, cudaGraphCreate(&graph, 0));
    auto fail_graph = [&](cudaError_t e, const char* what) {
        if (exec) cudaGraphExecDestroy(exec);
        cudaGraphDestroy(graph);
        return cuda_fail(c, e, what);
    };
    cudaGraphConditionalHandle handle;
    cudaError_t e = cudaGraphConditionalHandleCreate(&handle, graph, 1, cudaGraphCondAssignDefault);
    if (e != cudaSuccess) return fail_graph(e, "cudaGraphConditionalHandleCreate");
    // (the parameter union has members without default constructors: zeroed raw storage)
    alignas(cudaGraphNodeParams) unsigned char np_bytes[sizeof(cudaGraphNodeParams)];
    memset(np_bytes, 0, sizeof np_bytes);
    cudaGraphNodeParams* np = reinterpret_cast<cudaGraphNodeParams*>(np_bytes);
    np->type = cudaGraphNodeTypeConditional;
    np->conditional.handle = handle;
    np->conditional.type = cudaGraphCondTypeWhile;
    np->conditional.size = 1;
    cudaGraphNode_t node;
    e = cudaGraphAddNode(&node, graph, nullptr, nullptr, 0, np);
    if (e != cudaSuccess) return fail_graph(e, "cudaGraphAddNode (conditional)");
    cudaGraph_t body = np->conditional.phGraph_out[0];
    e = cudaStreamBeginCaptureToGraph(c->capture, body, nullptr, nullptr, 0, cudaStreamCaptureModeThreadLocal);
    if (e != cudaSuccess) return fail_graph(e, "cudaStreamBeginCaptureToGraph");
    const bool tracing = c->trace_on;
    c->trace_on = false;
    fr_status st = one_iteration(c->capture, -1);
    if (st == FR_OK) {
        cudaError_t ek = launch_converge(sq, static_cast<float*>(c->rmse.p), loop_iter,
                                         p->rule == FR_RULE_PAPER ? flame_cnt : nullptr, count_slots, iters,
                                         stop_delta, handle, c->capture);
        if (ek != cudaSuccess) st = cuda_fail(c, ek, "converge kernel");
    }
    c->trace_on = tracing;
    cudaGraph_t captured = nullptr;
    e = cudaStreamEndCapture(c->capture, &captured);
    if (st != FR_OK) {
        cudaGraphDestroy(graph);
        return st;
    }
    if (e != cudaSuccess) return fail_graph(e, "cudaStreamEndCapture");
    e = cudaGraphInstantiate(&exec, graph, 0);
    if (e != cudaSuccess) return fail_graph(e, "cudaGraphInstantiate");
    e = cudaGraphLaunch(exec, s);
    if (e != cudaSuccess) return fail_graph(e, "cudaGraphLaunch");
    int done = 0;
    e = cudaMemcpyAsync(c->host_counter, loop_iter, sizeof(int), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return fail_graph(e, "loop counter");
    cudaGraphExecDestroy(exec);
    cudaGraphDestroy(graph);
    loop_done();
    memcpy(&done, c->host_counter, sizeof(int));
    if (iters_done) *iters_done = done;
    if (rmse && done > 0) {
        FR_CUDA(c, cudaMemcpyAsync(rmse, c->rmse.p, (size_t)done * 12,
                                   rmse_is_host ? cudaMemcpyDeviceToHost : cudaMemcpyDeviceToDevice, s));
        if (rmse_is_host) FR_CUDA(c, cudaStreamSynchronize(s));
    }
    return FR_OK;
}

extern "C" fr_status fr_reconstruct(fr_ctx* c, fr_volume* vol, const float* albedo, const fr_camera* cams,
                                    int ncam, const float* targets, int targets_are_host, const int32_t* bbox,
                                    int iters, int first_iteration, const fr_params* p, float* rmse,
                                    int rmse_is_host)
{
    return reconstruct_impl(c, vol, albedo, cams, ncam, targets, targets_are_host, bbox, iters, first_iteration, p,
                            rmse, rmse_is_host, -1.0f, nullptr);
}

extern "C" fr_status fr_reconstruct_until(fr_ctx* c, fr_volume* vol, const float* albedo, const fr_camera* cams,
                                          int ncam, const float* targets, int targets_are_host,
                                          const int32_t* bbox, int max_iters, float stop_delta,
                                          int first_iteration, const fr_params* p, float* rmse, int rmse_is_host,
                                          int32_t* iters_done)
{
    if (!c) return FR_EINVAL;
    if (!(stop_delta >= 0.0f) || !std::isfinite(stop_delta))
        return fail(c, FR_EINVAL, "stop_delta must be finite and >= 0");
    if (!iters_done) return fail(c, FR_EINVAL, "iters_done is NULL");
    if (max_iters < 1) return fail(c, FR_EINVAL, "max_iters must be >= 1");
    *iters_done = 0;
    return reconstruct_impl(c, vol, albedo, cams, ncam, targets, targets_are_host, bbox, max_iters,
                            first_iteration, p, rmse, rmse_is_host, stop_delta, iters_done);
}

// ---------------------------------------------------------------------------
// Rendering with residual, without any allocation
// ---------------------------------------------------------------------------
//
// fr_render_residual keeps its per-CTA squared-error partials in scratch that
// the context allocates on first use.  Some callers cannot allocate device
// memory when they render: a process that hands all device memory to its own
// pool at start-up (a fresh cudaMalloc would fail or fragment that budget),
// or a latency-critical loop that forbids cudaMalloc/cudaFree after start-up
// because they can synchronise the whole device.  This variant keeps the
// partials in a fixed file-scope device array instead, so it allocates
// nothing, device or host.

// FR_NOALLOC_MAX_TILES tiles of 16 x 8 pixels (4 floats each, 1 MiB in
// total), held by every GPU that loads the library until the process exits.
static __device__ __align__(256) float g_noalloc_partials[4 * FR_NOALLOC_MAX_TILES];

namespace {

constexpr int kNoAllocMaxDevices = 64;
std::mutex g_noalloc_mu;
float* g_noalloc_ptr[kNoAllocMaxDevices] = {};

// Device address of g_noalloc_partials on `device`, looked up once per device
// with that device current.  In host code the array's name is only a host
// stand-in: kernels must be given this address.  The same one-time set-up
// loads every kernel the entry point launches: with lazy module loading (the
// default since CUDA 12) the array, the module and each kernel would
// otherwise be loaded -- taking device memory -- at their first use, which
// could fail in a process whose pool already holds all device memory.
fr_status noalloc_scratch(fr_ctx* c, int device, float** out)
{
    std::lock_guard<std::mutex> lock(g_noalloc_mu);
    if (!g_noalloc_ptr[device]) {
        int prev = 0;
        FR_CUDA(c, cudaGetDevice(&prev));
        FR_CUDA(c, cudaSetDevice(device));
        void* addr = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&addr, g_noalloc_partials);
        const char* what = "cudaGetSymbolAddress(g_noalloc_partials)";
        if (e == cudaSuccess) {
            e = preload_noalloc_kernels();
            what = "loading the render kernels";
        }
        cudaSetDevice(prev);
        if (e != cudaSuccess) return cuda_fail(c, e, what);
        g_noalloc_ptr[device] = static_cast<float*>(addr);
    }
    *out = g_noalloc_ptr[device];
    return FR_OK;
}

}  // namespace

extern "C" fr_status fr_render_residual_noalloc(int device, void* stream, const fr_volume* vol,
                                                const fr_camera* cams, int ncam, const fr_params* p,
                                                const float* targets, const int32_t* bbox, float* rendered,
                                                float* residual, float* sq_err, char* err, size_t err_len)
{
    fr_ctx c;  // stack context for validation messages; holds no resources
    c.device = device;
    c.stream = static_cast<cudaStream_t>(stream);
    auto done = [&](fr_status s) {
        if (err && err_len) snprintf(err, err_len, "%s", s == FR_OK ? "" : c.err);
        return s;
    };
    int ndev = 0;
    if (cudaGetDeviceCount(&ndev) != cudaSuccess) {
        cudaGetLastError();
        return done(fail(&c, FR_ECUDA, "no CUDA device"));
    }
    if (device < 0 || device >= ndev || device >= kNoAllocMaxDevices)
        return done(fail(&c, FR_EINVAL, "device %d out of range", device));
    fr_status s;
    if ((s = check_volume(&c, vol, "vol")) || (s = check_cams(&c, cams, ncam)) ||
        (s = check_params(&c, p, vol, cams)))
        return done(s);
    const int nt = tiles_of(cams[0].width, cams[0].height, ncam);
    if (nt > FR_NOALLOC_MAX_TILES)
        return done(fail(&c, FR_EINVAL,
                         "%d tiles of 16x8 pixels exceed the fixed scratch of %d tiles; use fr_render_residual",
                         nt, FR_NOALLOC_MAX_TILES));
    const size_t ib = image_bytes(cams, ncam);
    if ((s = check_dev(&c, targets, ib, "targets")) ||
        (s = check_dev(&c, bbox, (size_t)ncam * 4 * sizeof(int32_t), "bbox")) ||
        (rendered && (s = check_dev(&c, rendered, ib, "rendered"))) ||
        (s = check_dev(&c, residual, ib, "residual")) || (s = check_dev(&c, sq_err, 4 * sizeof(float), "sq_err")))
        return done(s);
    float* partials = nullptr;
    if ((s = noalloc_scratch(&c, device, &partials))) return done(s);
    int prev = 0;
    if (cudaGetDevice(&prev) != cudaSuccess || cudaSetDevice(device) != cudaSuccess)
        return done(cuda_fail(&c, cudaGetLastError(), "cudaSetDevice"));
    SingleArgs a;  // on the stack: no allocation
    fill_problem(vol, cams, ncam, p, a);
    a.p.targets = targets;
    a.p.bbox = bbox;
    a.p.rendered = rendered;
    a.p.residual = residual;
    a.p.partials = partials;  // every tile overwrites its own 4 floats: nothing to clear
    cudaError_t e = launch_fwd(a, vol->dtype, vol->kind, nt, c.stream);
    if (e == cudaSuccess) e = launch_finalize(partials, nt, sq_err, c.stream);
    cudaSetDevice(prev);
    if (e != cudaSuccess) return done(cuda_fail(&c, e, "launch"));
    return done(FR_OK);
}

// ---------------------------------------------------------------------------
// Batched reconstruction
// ---------------------------------------------------------------------------

extern "C" fr_status fr_reconstruct_batch(fr_ctx* c, const fr_problem* probs, int nprob, int iters,
                                          int first_iteration, const fr_params* p, int use_graph)
{
    FR_BEGIN(c);
    if (!probs || nprob < 1 || nprob > (1 << 20)) return fail(c, FR_EINVAL, "need 1 <= nprob <= 2^20");
    if (iters < 0) return fail(c, FR_EINVAL, "iters must be >= 0");
    if (first_iteration < 0 || (long long)first_iteration + iters > (1 << 20))
        return fail(c, FR_EINVAL, "iterations must stay below 2^20");
    if (!p) return fail(c, FR_EINVAL, "params is NULL");
    if (p->rule != FR_RULE_PAPER) return fail(c, FR_EINVAL, "batched reconstruction uses FR_RULE_PAPER");
    const int dt = probs[0].vol.dtype;
    // visual hull per problem (from its own targets) and exact empty-brick skipping
    const bool hull = p->use_hull != 0;
    const bool skip = p->skip_empty && !(p->tau > 0.0f);
    // the adjustment over ray parts (FR_BATCH_PARTS; whole rays by default)
    // when every problem's pixel index leaves the list entries' top two bits free
#if FR_BATCH_PARTS > 1
    int parts = FR_BATCH_PARTS;
    for (int i = 0; i < nprob; ++i) {
        const fr_problem& q = probs[i];
        if (q.cams && q.ncam > 0 && (long long)q.ncam * q.cams[0].width * q.cams[0].height >= (1LL << 30) - 1)
            parts = 1;
    }
#else
    const int parts = 1;
#endif
    // sizes and validation
    size_t arena = 0, cams_total = 0;
    long long tiles_total = 0;
    for (int i = 0; i < nprob; ++i) {
        const fr_problem& q = probs[i];
        char name[48];
        snprintf(name, sizeof name, "probs[%d].vol", i);
        FR_TRY(check_volume(c, &q.vol, name));
        if (q.vol.kind != FR_KIND_RGB || q.vol.dtype != dt)
            return fail(c, FR_EINVAL, "probs[%d]: batched volumes are RGB records of one storage type", i);
        FR_TRY(check_cams(c, q.cams, q.ncam));
        FR_TRY(check_params(c, p, &q.vol, q.cams));
        const size_t ib = image_bytes(q.cams, q.ncam);
        FR_TRY(check_dev(c, q.targets, ib, "targets"));
        FR_TRY(check_dev(c, q.bbox, (size_t)q.ncam * 16, "bbox"));
        if (q.rmse) FR_TRY(check_dev(c, q.rmse, (size_t)iters * 12, "rmse"));
        if (hull && q.hull_tags) FR_TRY(check_dev(c, q.hull_tags, (size_t)node_count(&q.vol) * 4, "hull_tags"));
        const long long npix = (long long)q.ncam * q.cams[0].width * q.cams[0].height;
        if (npix >= (1LL << 32)) return fail(c, FR_EINVAL, "probs[%d]: at most 2^32 pixels", i);
        const int nt = tiles_of(q.cams[0].width, q.cams[0].height, q.ncam);
        arena += align256(ib) + align256((size_t)node_count(&q.vol) * 16) + align256((size_t)nt * 16) +
                 align256((size_t)std::max(iters, 1) * 16) + align256(flame_list_buf_entries(nt) * 4) +
                 align256((size_t)nt * kTileThreads * 4 * parts) +
                 align256((size_t)node_count(&q.vol) * 2 * rec_bytes(&q.vol)) +
                 align256((size_t)npix * 4 * (parts - 1));
        const size_t tb = align256(brick_table_bytes(q.vol.nx, q.vol.ny, q.vol.nz));
        if (hull) arena += align256((size_t)node_count(&q.vol) * 4);
        if (skip) arena += tb;
        if (hull && skip) arena += tb;
        tiles_total += nt;
        cams_total += (size_t)q.ncam;
    }
    if (tiles_total * parts >= (1LL << 31)) return fail(c, FR_EINVAL, "too many tiles in one batch");
    if (iters == 0) return FR_OK;
    // ray weight tables for every problem (fr_params.tables, as in
    // fr_reconstruct), or for none when one of them has no room
    bool tabled = !FR_FUSED && p->tables != 1 && hull && skip && !(p->g_std > 0.0f) &&
                  (p->tables == 2 || iters >= FR_TABLES_MIN_ITERS);
    const size_t tab_probs = align256(sizeof(ProbDev) * nprob);
    const size_t tab_cams = align256(sizeof(CamDev) * cams_total);
    const size_t tab_tiles = align256(sizeof(int) * (nprob + 1));
    const size_t tab_blks = align256(sizeof(int) * (nprob + 1));
    const size_t tab_its = align256(sizeof(TabIter) * nprob);
    const size_t rmse_all = align256(sizeof(float) * 3 * (size_t)nprob * iters);
    const size_t tables = tab_probs + tab_cams + tab_tiles + tab_blks + tab_its;
    FR_TRY(ensure(c, c->batch, arena + tables + rmse_all, "batch"));
    // host staging (pinned), reused once the previous copy out of it is done
    if (!c->staging_done) FR_CUDA(c, cudaEventCreateWithFlags(&c->staging_done, cudaEventDisableTiming));
    FR_CUDA(c, cudaEventSynchronize(c->staging_done));
    if (c->staging_bytes < tables) {
        if (c->staging) cudaFreeHost(c->staging);
        c->staging = nullptr;
        c->staging_bytes = 0;
        if (cudaMallocHost(&c->staging, tables) != cudaSuccess) {
            cudaGetLastError();
            return fail(c, FR_ENOMEM, "cannot allocate %zu bytes of pinned staging", tables);
        }
        c->staging_bytes = tables;
    }
    char* dbase = static_cast<char*>(c->batch.p);
    ProbDev* d_probs = reinterpret_cast<ProbDev*>(dbase + arena);
    CamDev* d_cams = reinterpret_cast<CamDev*>(dbase + arena + tab_probs);
    int* d_tiles = reinterpret_cast<int*>(dbase + arena + tab_probs + tab_cams);
    float* d_rmse = reinterpret_cast<float*>(dbase + arena + tables);
    ProbDev* h_probs = reinterpret_cast<ProbDev*>(c->staging);
    CamDev* h_cams = reinterpret_cast<CamDev*>(static_cast<char*>(c->staging) + tab_probs);
    int* h_tiles = reinterpret_cast<int*>(static_cast<char*>(c->staging) + tab_probs + tab_cams);
    int* d_blks = reinterpret_cast<int*>(dbase + arena + tab_probs + tab_cams + tab_tiles);
    int* h_blks = reinterpret_cast<int*>(static_cast<char*>(c->staging) + tab_probs + tab_cams + tab_tiles);
    TabIter* d_its = reinterpret_cast<TabIter*>(dbase + arena + tab_probs + tab_cams + tab_tiles + tab_blks);
    TabIter* h_its =
        reinterpret_cast<TabIter*>(static_cast<char*>(c->staging) + tab_probs + tab_cams + tab_tiles + tab_blks);
    if (tabled && c->tab_batch.size() < 2 * (size_t)nprob) c->tab_batch.resize(2 * (size_t)nprob);
    fr_status tab_status = FR_OK;
    cudaStream_t s = c->stream;
    static thread_local SingleArgs a;
    size_t off = 0, cam_off = 0;
    int tile_off = 0;
    for (int i = 0; i < nprob; ++i) {
        const fr_problem& q = probs[i];
        fill_problem(&q.vol, q.cams, q.ncam, p, a);
        const int nt = tiles_of(q.cams[0].width, q.cams[0].height, q.ncam);
        const long long nodes = node_count(&q.vol);
        const size_t ib = image_bytes(q.cams, q.ncam);
        float* residual = reinterpret_cast<float*>(dbase + off); off += align256(ib);
        float* dV = reinterpret_cast<float*>(dbase + off); off += align256((size_t)nodes * 16);
        float* partials = reinterpret_cast<float*>(dbase + off); off += align256((size_t)nt * 16);
        float* sqerr = reinterpret_cast<float*>(dbase + off); off += align256((size_t)iters * 16);
        unsigned* fbuf = reinterpret_cast<unsigned*>(dbase + off); off += align256(flame_list_buf_entries(nt) * 4);
        // (runs padded to whole warps: at most a tile's worth of entries per tile and part)
        unsigned* flist = reinterpret_cast<unsigned*>(dbase + off);
        off += align256((size_t)nt * kTileThreads * 4 * parts);
        void* pairs = dbase + off; off += align256((size_t)nodes * 2 * rec_bytes(&q.vol));
        const size_t npix_q = (size_t)q.ncam * q.cams[0].width * q.cams[0].height;
        float* tpart = parts > 1 ? reinterpret_cast<float*>(dbase + off) : nullptr;
        off += align256(npix_q * 4 * (parts - 1));
        const size_t tb = align256(brick_table_bytes(q.vol.nx, q.vol.ny, q.vol.nz));
        unsigned* tags = nullptr;
        unsigned char *occ = nullptr, *hb = nullptr;
        if (hull) { tags = reinterpret_cast<unsigned*>(dbase + off); off += align256((size_t)nodes * 4); }
        if (skip) { occ = reinterpret_cast<unsigned char*>(dbase + off); off += tb; }
        if (hull && skip) { hb = reinterpret_cast<unsigned char*>(dbase + off); off += tb; }
        const int nbx = bricks_along(q.vol.nx), nby = bricks_along(q.vol.ny), nbz = bricks_along(q.vol.nz);
        const unsigned full = q.ncam >= 32 ? 0xffffffffu : ((1u << q.ncam) - 1u);
        if (hull) {
            // the problem's own tags when given, else its hull from its targets
            if (q.hull_tags) tags = const_cast<unsigned*>(reinterpret_cast<const unsigned*>(q.hull_tags));
            else FR_TRY(hull_tags(c, a, q.targets, p->flame_thresh, tags));
            FR_CUDA(c, launch_hull_clear(q.vol.data, dt, q.vol.nx, q.vol.ny, q.vol.nz, tags, full, hb, s));
        }
        ProbDev& P = a.p;
        P.nbx = nbx;
        P.nby = nby;
        P.nbz = nbz;
        P.occ = occ;
        P.occ_box = occ ? brick_box(occ, nbx, nby, nbz) : nullptr;
        P.hull = tags;
        P.hull_full = full;
        P.adj_occ = hb;
        P.adj_box = hb ? brick_box(hb, nbx, nby, nbz) : nullptr;
        // ray parts divide the samples inside the hull's box (see fr_reconstruct)
        P.split_box = FR_SPLIT_BOX && FR_BATCH_PARTS > 1 && hb && !(p->tau > 0.0f) ? 1 : 0;
        P.cams = d_cams + cam_off;
        P.targets = q.targets;
        P.bbox = q.bbox;
        P.residual = residual;
        P.partials = partials;
        P.dV = dV;
        P.img_in = residual;
        P.img_scale = 1.0f;
        P.list = flist;
        P.list_count = fbuf + flame_list_total_at(nt);
        P.vol_rw = q.vol.data;
        P.nodes = nodes;
        P.sqerr = sqerr;
        P.ntiles = nt;
        P.iteration = first_iteration;
        P.sq_slot = 0;
        P.pairs = pairs;
        P.tpart = tpart;
        if (tabled) {
            // the problem's tables in its own two context buffers
            TabMemory mem;
            mem.status = &tab_status;
            Buf* tb = &c->tab_batch[2 * (size_t)i];
            mem.scratch = [c, tb, &tab_status](size_t n) -> void* {
                tab_status = ensure(c, tb[0], n, "batch table counts");
                if (tab_status == FR_ENOMEM) c->err[0] = '\0';
                return tab_status == FR_OK ? tb[0].p : nullptr;
            };
            mem.tables = [c, tb, &tab_status](size_t n) -> void* {
                tab_status = ensure(c, tb[1], n, "batch ray weight tables");
                if (tab_status == FR_ENOMEM) c->err[0] = '\0';
                return tab_status == FR_OK ? tb[1].p : nullptr;
            };
            bool built = false;
            a.p.adj_occ = hb;
            a.p.adj_box = P.adj_box;
            a.p.nbx = nbx;
            a.p.nby = nby;
            a.p.nbz = nbz;
            a.p.targets = q.targets;
            FR_TRY(build_tables(c, a, &q.vol, tags, full, nt, mem, h_its[i], built));
            if (!built) tabled = false;
            h_blks[i] = i ? h_blks[i - 1] + (int)tab_adjust_blocks(h_its[i - 1].nhull) : 0;
        }
        h_probs[i] = P;
        for (int v = 0; v < q.ncam; ++v) h_cams[cam_off + v] = a.cams[v];
        h_tiles[i] = tile_off;
        FR_CUDA(c, cudaMemsetAsync(dV, 0, (size_t)nodes * 16, s));
        FR_CUDA(c, launch_flame_list(a, nt, fbuf, flist, s, parts));
        cam_off += (size_t)q.ncam;
        tile_off += nt;
    }
    h_tiles[nprob] = tile_off;
    int blk_total = 0;
    if (tabled) {
        blk_total = h_blks[nprob - 1] + (int)tab_adjust_blocks(h_its[nprob - 1].nhull);
        h_blks[nprob] = blk_total;
        // the first iteration's staged records; the residual images are not needed
        for (int i = 0; i < nprob; ++i) {
            FR_CUDA(c, launch_tab_stage(probs[i].vol.data, dt, h_its[i], s));
            h_probs[i].residual = nullptr;
        }
    }
    FR_CUDA(c, cudaMemcpyAsync(d_probs, h_probs, tables, cudaMemcpyHostToDevice, s));
    FR_CUDA(c, cudaEventRecord(c->staging_done, s));
    const bool tau = p->tau > 0.0f;

    auto iterate = [&](cudaStream_t st) -> cudaError_t {
        cudaError_t e = cudaSuccess;
        for (int it = 0; it < iters && e == cudaSuccess && tabled; ++it) {
            // rendering from the forward tables, error sums, the adjustment
            // tables' update (which stages the next iteration's records)
            e = launch_tab_forward_batch(d_probs, d_its, d_tiles, nprob, tile_off, dt, st);
            if (e == cudaSuccess) e = launch_finalize_batch(d_probs, nprob, it, st);
            if (e == cudaSuccess)
                e = launch_tab_adjust_batch(d_probs, d_its, d_blks, nprob, blk_total, dt, p->clamp_nonneg, st);
        }
        for (int it = 0; it < iters && e == cudaSuccess && !tabled; ++it) {
            if (skip) e = launch_brick_reset_batch(d_probs, nprob, st);
            if (e == cudaSuccess) e = launch_pair_pack_batch(d_probs, nprob, dt, st);
            if (e == cudaSuccess && skip) e = launch_brick_box_batch(d_probs, nprob, st);
            if (e == cudaSuccess)
                e = launch_fwd_batch(d_probs, d_tiles, nprob, tile_off, dt, KIND_RGB, tau, true, st, skip);
            if (e == cudaSuccess) e = launch_finalize_batch(d_probs, nprob, it, st);
            if (e == cudaSuccess)
                e = launch_adjust_list_batch(d_probs, d_tiles, nprob, tile_off, dt, tau, it, st, hull && skip, parts);
            if (e == cudaSuccess) e = launch_apply_batch(d_probs, nprob, dt, p->clamp_nonneg, st);   // + hull clear
        }
        return e;
    };
    if (use_graph) {
        if (!c->capture) FR_CUDA(c, cudaStreamCreateWithFlags(&c->capture, cudaStreamNonBlocking));
        cudaGraph_t graph = nullptr;
        cudaGraphExec_t exec = nullptr;
        FR_CUDA(c, cudaStreamBeginCapture(c->capture, cudaStreamCaptureModeThreadLocal));
        cudaError_t e = iterate(c->capture);
        cudaError_t e2 = cudaStreamEndCapture(c->capture, &graph);
        if (e != cudaSuccess || e2 != cudaSuccess) {
            if (graph) cudaGraphDestroy(graph);
            return cuda_fail(c, e != cudaSuccess ? e : e2, "graph capture");
        }
        e = cudaGraphInstantiate(&exec, graph, 0);
        cudaGraphDestroy(graph);
        if (e != cudaSuccess) return cuda_fail(c, e, "cudaGraphInstantiate");
        e = cudaGraphLaunch(exec, s);
        cudaError_t e3 = cudaStreamSynchronize(s);
        cudaGraphExecDestroy(exec);
        if (e != cudaSuccess) return cuda_fail(c, e, "cudaGraphLaunch");
        if (e3 != cudaSuccess) return cuda_fail(c, e3, "cudaStreamSynchronize");
    } else {
        FR_CUDA(c, iterate(s));
    }
    FR_CUDA(c, launch_rmse_batch(d_probs, nprob, iters, d_rmse, s));
    for (int i = 0; i < nprob; ++i)
        if (probs[i].rmse)
            FR_CUDA(c, cudaMemcpyAsync(probs[i].rmse, d_rmse + (size_t)3 * iters * i, (size_t)iters * 12,
                                       cudaMemcpyDeviceToDevice, s));
    return FR_OK;
}
