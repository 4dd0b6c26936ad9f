// server.cu -- continuous-batching reconstruction server over the batched
// kernels: admission by device-memory budget, one iteration of every
// resident job per step in shared launches, retirement at step boundaries.
#include <chrono>
#include <deque>
#include <vector>

#include "abi_common.h"

struct fr_job {
    fr_job_desc d;
    std::vector<fr_camera> cams;
    int state = FR_JOB_QUEUED;
    int iters_done = 0;
    bool cancel = false;
    size_t footprint = 0;
    double t_submit = 0.0, t_admit = 0.0, t_done = 0.0;
    // device memory while resident (one pool allocation)
    char* mem = nullptr;
    void* vol = nullptr;
    float* targets = nullptr;
    int* bbox = nullptr;
    float* residual = nullptr;
    float* dV = nullptr;
    float* partials = nullptr;
    float* sqerr = nullptr;
    unsigned* fbuf = nullptr;
    unsigned* flist = nullptr;
    float* tpart = nullptr;             // transmittance at the ray parts' starts (flame pixels)
    void* pairs = nullptr;
    unsigned* tags = nullptr;           // visual hull tags (server with use_hull)
    unsigned char* occ = nullptr;       // brick table of the non-empty records (skip_empty)
    unsigned char* hull_bricks = nullptr;  // brick table of the hull (both)
    int ntiles = 0;
    // ray weight tables (the paper rule in the visual hull with skipping, field
    // mode, G = 1, jobs of FR_TABLES_MIN_ITERS iterations or more): built at
    // admission in two more pool allocations, counted in the footprint
    bool tabled = false;
    TabIter tab{};
    void* tab_scratch = nullptr;
    void* tab_block = nullptr;
};

struct fr_server {
    fr_ctx* ctx = nullptr;
    fr_params p{};
    int dtype = FR_F32;
    size_t budget = 0, used = 0;
    cudaMemPool_t pool = nullptr;
    std::deque<fr_job*> queue;
    std::vector<fr_job*> resident;
    Buf tables;                  // device ProbDev / CamDev / tile starts
    void* staging = nullptr;     // pinned host staging of the tables
    size_t staging_bytes = 0;
    cudaEvent_t staging_done = nullptr;
    std::chrono::steady_clock::time_point t0;

    double now() const
    {
        return std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
    }
};

namespace {

struct JobLayout {
    size_t vol, targets, bbox, residual, dV, partials, sqerr, fbuf, flist, tpart, pairs, tags, occ, hull_bricks, total;
};

// Parts each flame ray is adjusted in (FR_BATCH_PARTS, whole rays by
// default); with parts the list entries carry the part in their top two bits,
// so jobs stay below 2^30 - 1 pixels (fr_server_submit refuses larger ones).
constexpr int kServerParts = FR_BATCH_PARTS;

bool server_hull(const fr_server* s) { return s->p.use_hull != 0; }
bool server_skip(const fr_server* s) { return s->p.skip_empty && !(s->p.tau > 0.0f); }

JobLayout job_layout(const fr_job_desc& d, int dtype, const fr_camera* cams, bool hull, bool skip)
{
    JobLayout L{};
    const long long nodes = (long long)d.nx * d.ny * d.nz;
    const size_t ib = image_bytes(cams, d.ncam);
    const int nt = tiles_of(cams[0].width, cams[0].height, d.ncam);
    size_t o = 0;
    L.vol = o; o += align256((size_t)nodes * 4 * dtype_bytes(dtype));
    L.targets = o; o += align256(ib);
    L.bbox = o; o += align256((size_t)d.ncam * 16);
    L.residual = o; o += align256(ib);
    L.dV = o; o += align256((size_t)nodes * 16);
    L.partials = o; o += align256((size_t)nt * 16);
    L.sqerr = o; o += align256((size_t)std::max(d.iters, 1) * 16);
    L.fbuf = o; o += align256(flame_list_buf_entries(nt) * 4);
    L.flist = o; o += align256((size_t)nt * kTileThreads * 4 * kServerParts);   // runs padded to whole warps
    L.tpart = o; o += align256((size_t)d.ncam * cams[0].width * cams[0].height * 4 * (kServerParts - 1));
    L.pairs = o; o += align256((size_t)nodes * 8 * dtype_bytes(dtype));
    const size_t tb = align256(brick_table_bytes(d.nx, d.ny, d.nz));
    L.tags = o; if (hull) o += align256((size_t)nodes * 4);
    L.occ = o; if (skip) o += tb;
    L.hull_bricks = o; if (hull && skip) o += tb;
    L.total = o;
    return L;
}

fr_volume job_volume(const fr_job* j, int dtype)
{
    fr_volume v{};
    v.nx = j->d.nx; v.ny = j->d.ny; v.nz = j->d.nz;
    v.kind = FR_KIND_RGB;
    v.dtype = dtype;
    for (int a = 0; a < 3; ++a) v.origin[a] = j->d.origin[a];
    v.h = j->d.h;
    v.data = j->vol;
    return v;
}

void job_free(fr_server* s, fr_job* j)
{
    for (void** p : {&j->tab_scratch, &j->tab_block})
        if (*p) {
            cudaFreeAsync(*p, s->ctx->stream);
            *p = nullptr;
        }
    j->tabled = false;
    if (j->mem) {
        cudaFreeAsync(j->mem, s->ctx->stream);
        j->mem = nullptr;
        s->used -= j->footprint;
    }
}

// Whether a job builds ray weight tables (fr_params.tables of the server).
bool server_tables(const fr_server* s, const fr_job* j)
{
    const fr_params& p = s->p;
    return !FR_FUSED && p.tables != 1 && p.rule == FR_RULE_PAPER && p.use_hull && p.skip_empty && !(p.tau > 0.0f) &&
           !(p.g_std > 0.0f) && (p.tables == 2 || j->d.iters >= FR_TABLES_MIN_ITERS);
}

// A pool allocation for a job's tables inside the server's budget (nullptr
// and *st = FR_ENOMEM when there is no room); counted in the job's footprint.
void* job_tab_alloc(fr_server* s, fr_job* j, size_t n, void** slot, fr_status* st)
{
    if (s->used + n > s->budget) {
        *st = FR_ENOMEM;
        return nullptr;
    }
    void* p = nullptr;
    if (cudaMallocFromPoolAsync(&p, n, s->pool, s->ctx->stream) != cudaSuccess) {
        cudaGetLastError();
        *st = FR_ENOMEM;
        return nullptr;
    }
    *slot = p;
    s->used += n;
    j->footprint += n;
    return p;
}

// Admission: allocate, upload the initial volume and the frames, prepare the
// targets and build the flame-ray list.
fr_status job_admit(fr_server* s, fr_job* j)
{
    fr_ctx* c = s->ctx;
    cudaStream_t st = c->stream;
    const bool hull = server_hull(s), skip = server_skip(s);
    const JobLayout L = job_layout(j->d, s->dtype, j->cams.data(), hull, skip);
    void* mem = nullptr;
    cudaError_t e = cudaMallocFromPoolAsync(&mem, L.total, s->pool, st);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return fail(c, FR_ENOMEM, "job %p: device allocation of %zu bytes failed", (void*)j, L.total);
    }
    j->mem = static_cast<char*>(mem);
    s->used += j->footprint;
    j->vol = j->mem + L.vol;
    j->targets = reinterpret_cast<float*>(j->mem + L.targets);
    j->bbox = reinterpret_cast<int*>(j->mem + L.bbox);
    j->residual = reinterpret_cast<float*>(j->mem + L.residual);
    j->dV = reinterpret_cast<float*>(j->mem + L.dV);
    j->partials = reinterpret_cast<float*>(j->mem + L.partials);
    j->sqerr = reinterpret_cast<float*>(j->mem + L.sqerr);
    j->fbuf = reinterpret_cast<unsigned*>(j->mem + L.fbuf);
    j->flist = reinterpret_cast<unsigned*>(j->mem + L.flist);
    j->tpart = kServerParts > 1 ? reinterpret_cast<float*>(j->mem + L.tpart) : nullptr;
    j->pairs = j->mem + L.pairs;
    j->tags = hull ? reinterpret_cast<unsigned*>(j->mem + L.tags) : nullptr;
    j->occ = skip ? reinterpret_cast<unsigned char*>(j->mem + L.occ) : nullptr;
    j->hull_bricks = hull && skip ? reinterpret_cast<unsigned char*>(j->mem + L.hull_bricks) : nullptr;
    const long long nodes = (long long)j->d.nx * j->d.ny * j->d.nz;
    const size_t ib = image_bytes(j->cams.data(), j->d.ncam);
    const int W = j->cams[0].width, H = j->cams[0].height;
    j->ntiles = tiles_of(W, H, j->d.ncam);
    FR_CUDA(c, cudaMemcpyAsync(j->vol, j->d.init_records, (size_t)nodes * 4 * dtype_bytes(s->dtype),
                               cudaMemcpyHostToDevice, st));
    FR_CUDA(c, cudaMemcpyAsync(j->targets, j->d.targets, ib, cudaMemcpyHostToDevice, st));
    FR_CUDA(c, cudaMemsetAsync(j->dV, 0, (size_t)nodes * 16, st));
    FR_CUDA(c, launch_prepare_targets(j->targets, j->d.ncam, H, W, s->p.flame_thresh, j->bbox, st));
    static thread_local SingleArgs a;
    fr_volume v = job_volume(j, s->dtype);
    fill_problem(&v, j->cams.data(), j->d.ncam, &s->p, a);
    a.p.targets = j->targets;
    FR_CUDA(c, launch_flame_list(a, j->ntiles, j->fbuf, j->flist, st, kServerParts));
    if (hull) {
        // the job's visual hull from its prepared frames; records outside it cleared
        const unsigned full = j->d.ncam >= 32 ? 0xffffffffu : ((1u << j->d.ncam) - 1u);
        if (j->d.hull_tags)
            FR_CUDA(c, cudaMemcpyAsync(j->tags, j->d.hull_tags, (size_t)nodes * 4, cudaMemcpyHostToDevice, st));
        else
            FR_TRY(hull_tags(c, a, j->targets, s->p.flame_thresh, j->tags));
        FR_CUDA(c, launch_hull_clear(j->vol, s->dtype, j->d.nx, j->d.ny, j->d.nz, j->tags, full, j->hull_bricks, st));
        if (j->hull_bricks && server_tables(s, j)) {
            // the job's tables, then its first iteration's staged records
            if (j->d.alpha_l != 0.0f) a.p.alpha_l = j->d.alpha_l;
            a.p.nbx = bricks_along(j->d.nx);
            a.p.nby = bricks_along(j->d.ny);
            a.p.nbz = bricks_along(j->d.nz);
            a.p.adj_occ = j->hull_bricks;
            a.p.adj_box = brick_box(j->hull_bricks, a.p.nbx, a.p.nby, a.p.nbz);
            fr_status ms = FR_OK;
            TabMemory mem;
            mem.status = &ms;
            mem.scratch = [s, j, &ms](size_t n) { return job_tab_alloc(s, j, n, &j->tab_scratch, &ms); };
            mem.tables = [s, j, &ms](size_t n) { return job_tab_alloc(s, j, n, &j->tab_block, &ms); };
            bool built = false;
            FR_TRY(build_tables(c, a, &v, j->tags, full, j->ntiles, mem, j->tab, built));
            if (built) {
                FR_CUDA(c, launch_tab_stage(j->vol, s->dtype, j->tab, st));
                j->tabled = true;
            } else {
                // (no room: the job marches; what the build took goes back)
                for (void** p : {&j->tab_scratch, &j->tab_block})
                    if (*p) {
                        cudaFreeAsync(*p, st);
                        *p = nullptr;
                    }
                const size_t extra = j->footprint - job_layout(j->d, s->dtype, j->cams.data(), hull, skip).total;
                s->used -= extra;
                j->footprint -= extra;
            }
        }
    }
    j->state = FR_JOB_RUNNING;
    j->t_admit = s->now();
    return FR_OK;
}

// Completion: per-iteration error and the final volume back to the host.
fr_status job_complete(fr_server* s, fr_job* j)
{
    fr_ctx* c = s->ctx;
    cudaStream_t st = c->stream;
    const long long nodes = (long long)j->d.nx * j->d.ny * j->d.nz;
    if (j->d.rmse) {
        std::vector<float> sq((size_t)j->d.iters * 4);
        FR_CUDA(c, cudaMemcpyAsync(sq.data(), j->sqerr, sq.size() * 4, cudaMemcpyDeviceToHost, st));
        FR_CUDA(c, cudaStreamSynchronize(st));
        for (int i = 0; i < j->d.iters; ++i)
            for (int ch = 0; ch < 3; ++ch) {
                const float cnt = sq[4 * i + 3];
                j->d.rmse[3 * i + ch] = cnt > 0.0f ? 255.0f * std::sqrt(sq[4 * i + ch] / cnt) : 0.0f;
            }
    }
    FR_CUDA(c, cudaMemcpyAsync(j->d.result_records, j->vol, (size_t)nodes * 4 * dtype_bytes(s->dtype),
                               cudaMemcpyDeviceToHost, st));
    FR_CUDA(c, cudaStreamSynchronize(st));
    job_free(s, j);
    j->state = FR_JOB_DONE;
    j->t_done = s->now();
    return FR_OK;
}

}  // namespace

extern "C" fr_status fr_server_create(fr_ctx* c, const fr_params* p, int dtype, size_t budget, fr_server** out)
{
    FR_BEGIN(c);
    if (!out || !p) return fail(c, FR_EINVAL, "NULL argument");
    *out = nullptr;
    if (dtype != FR_F32 && dtype != FR_BF16 && dtype != FR_F16) return fail(c, FR_EINVAL, "bad dtype");
    if (p->rule != FR_RULE_PAPER) return fail(c, FR_EINVAL, "the server runs the paper rule");
    if (!(p->step > 0.0f) || !std::isfinite(p->alpha_l) || !(p->tau < 1.0f))
        return fail(c, FR_EINVAL, "bad parameters");
    size_t free_b = 0, total_b = 0;
    FR_CUDA(c, cudaMemGetInfo(&free_b, &total_b));
    if (budget == 0) budget = free_b / 10 * 8;
    if (budget > free_b) return fail(c, FR_ENOMEM, "budget %zu exceeds free device memory %zu", budget, free_b);
    fr_server* s = new (std::nothrow) fr_server();
    if (!s) return fail(c, FR_ENOMEM, "host allocation failed");
    s->ctx = c;
    s->p = *p;
    s->dtype = dtype;
    s->budget = budget;
    s->t0 = std::chrono::steady_clock::now();
    cudaMemPoolProps props{};
    props.allocType = cudaMemAllocationTypePinned;
    props.location.type = cudaMemLocationTypeDevice;
    props.location.id = c->device;
    cudaError_t e = cudaMemPoolCreate(&s->pool, &props);
    if (e == cudaSuccess) {
        uint64_t keep = UINT64_MAX;  // keep released memory in the pool between jobs
        e = cudaMemPoolSetAttribute(s->pool, cudaMemPoolAttrReleaseThreshold, &keep);
    }
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&s->staging_done, cudaEventDisableTiming);
    if (e != cudaSuccess) {
        cudaGetLastError();
        if (s->pool) cudaMemPoolDestroy(s->pool);
        delete s;
        return cuda_fail(c, e, "server set-up");
    }
    *out = s;
    return FR_OK;
}

extern "C" fr_status fr_server_destroy(fr_server* s)
{
    if (!s) return FR_EINVAL;
    fr_ctx* c = s->ctx;
    cudaSetDevice(c->device);
    cudaStreamSynchronize(c->stream);
    for (fr_job* j : s->resident) job_free(s, j);
    cudaStreamSynchronize(c->stream);
    if (s->tables.p) cudaFree(s->tables.p);
    if (s->staging) cudaFreeHost(s->staging);
    if (s->staging_done) cudaEventDestroy(s->staging_done);
    if (s->pool) cudaMemPoolDestroy(s->pool);
    delete s;
    return FR_OK;
}

extern "C" fr_status fr_server_submit(fr_server* s, const fr_job_desc* d, fr_job** out)
{
    if (!s) return FR_EINVAL;
    fr_ctx* c = s->ctx;
    FR_BEGIN(c);
    if (!d || !out) return fail(c, FR_EINVAL, "NULL argument");
    *out = nullptr;
    fr_volume v{};
    v.nx = d->nx; v.ny = d->ny; v.nz = d->nz;
    v.kind = FR_KIND_RGB;
    v.dtype = s->dtype;
    for (int a = 0; a < 3; ++a) v.origin[a] = d->origin[a];
    v.h = d->h;
    if (v.nx < 2 || v.ny < 2 || v.nz < 2 || v.nx > 8192 || v.ny > 8192 || v.nz > 8192)
        return fail(c, FR_EINVAL, "job extents must be in [2, 8192]");
    if (!(v.h > 0.0f) || !finite3(v.origin)) return fail(c, FR_EINVAL, "job spacing must be positive");
    FR_TRY(check_cams(c, d->cams, d->ncam));
    FR_TRY(check_params(c, &s->p, &v, d->cams));
    if (d->iters < 1 || d->iters > (1 << 20)) return fail(c, FR_EINVAL, "iters must be in [1, 2^20]");
    if (!std::isfinite(d->alpha_l)) return fail(c, FR_EINVAL, "alpha_l must be finite");
    if (!d->init_records || !d->targets || !d->result_records) return fail(c, FR_EINVAL, "NULL host buffer");
    const long long npix = (long long)d->ncam * d->cams[0].width * d->cams[0].height;
    if (npix >= (1LL << 30) - 1) return fail(c, FR_EINVAL, "at most 2^30 - 2 pixels per job");
    const size_t fp = job_layout(*d, s->dtype, d->cams, server_hull(s), server_skip(s)).total;
    if (fp > s->budget) return fail(c, FR_ENOMEM, "job needs %zu bytes, the budget is %zu", fp, s->budget);
    fr_job* j = new (std::nothrow) fr_job();
    if (!j) return fail(c, FR_ENOMEM, "host allocation failed");
    j->d = *d;
    j->cams.assign(d->cams, d->cams + d->ncam);
    j->d.cams = j->cams.data();
    j->footprint = fp;
    j->t_submit = s->now();
    s->queue.push_back(j);
    *out = j;
    return FR_OK;
}

extern "C" fr_status fr_server_step(fr_server* s, int* running, int* queued)
{
    if (!s) return FR_EINVAL;
    fr_ctx* c = s->ctx;
    FR_BEGIN(c);
    cudaStream_t st = c->stream;
    // retire cancelled jobs
    for (size_t i = 0; i < s->resident.size();) {
        fr_job* j = s->resident[i];
        if (j->cancel) {
            job_free(s, j);
            j->state = FR_JOB_CANCELED;
            j->t_done = s->now();
            s->resident.erase(s->resident.begin() + i);
        } else {
            ++i;
        }
    }
    // admit in arrival order while the budget allows
    while (!s->queue.empty()) {
        fr_job* j = s->queue.front();
        if (j->cancel) {
            s->queue.pop_front();
            j->state = FR_JOB_CANCELED;
            j->t_done = s->now();
            continue;
        }
        if (s->used + j->footprint > s->budget) break;
        s->queue.pop_front();
        fr_status r = job_admit(s, j);
        if (r != FR_OK) {
            // what the admission took goes back to the pool and the budget
            job_free(s, j);
            j->state = FR_JOB_CANCELED;
            j->t_done = s->now();
            return r;
        }
        s->resident.push_back(j);
    }
    const int n = (int)s->resident.size();
    if (n > 0) {
        // the resident jobs with tables first, then the marching ones
        std::vector<fr_job*> order;
        order.reserve(n);
        for (fr_job* j : s->resident)
            if (j->tabled) order.push_back(j);
        const int ntab = (int)order.size(), nm = n - ntab;
        for (fr_job* j : s->resident)
            if (!j->tabled) order.push_back(j);
        // tables of the resident jobs, with each job's own iteration
        size_t ncam = 0;
        for (fr_job* j : order) ncam += (size_t)j->d.ncam;
        const size_t tp = align256(sizeof(ProbDev) * n), tc = align256(sizeof(CamDev) * ncam);
        const size_t tt = align256(sizeof(int) * (nm + 1)), ttt = align256(sizeof(int) * (ntab + 1));
        const size_t tbs = align256(sizeof(int) * (ntab + 1)), tit = align256(sizeof(TabIter) * (ntab + 1));
        const size_t tables = tp + tc + tt + ttt + tbs + tit;
        FR_TRY(ensure(c, s->tables, tables, "server tables"));
        FR_CUDA(c, cudaEventSynchronize(s->staging_done));
        if (s->staging_bytes < tables) {
            if (s->staging) cudaFreeHost(s->staging);
            s->staging = nullptr;
            s->staging_bytes = 0;
            if (cudaMallocHost(&s->staging, tables * 2) != cudaSuccess) {
                cudaGetLastError();
                return fail(c, FR_ENOMEM, "pinned staging");
            }
            s->staging_bytes = tables * 2;
        }
        char* hb = static_cast<char*>(s->staging);
        char* db = static_cast<char*>(s->tables.p);
        ProbDev* hp = reinterpret_cast<ProbDev*>(hb);
        CamDev* hc = reinterpret_cast<CamDev*>(hb + tp);
        int* ht = reinterpret_cast<int*>(hb + tp + tc);                      // marching jobs' tile starts
        int* htt = reinterpret_cast<int*>(hb + tp + tc + tt);                // tabled jobs' tile starts
        int* hbs = reinterpret_cast<int*>(hb + tp + tc + tt + ttt);          // tabled jobs' adjustment blocks
        TabIter* hit = reinterpret_cast<TabIter*>(hb + tp + tc + tt + ttt + tbs);
        ProbDev* dp = reinterpret_cast<ProbDev*>(db);
        CamDev* dc = reinterpret_cast<CamDev*>(db + tp);
        int* dtl = reinterpret_cast<int*>(db + tp + tc);
        int* dtt = reinterpret_cast<int*>(db + tp + tc + tt);
        int* dbs = reinterpret_cast<int*>(db + tp + tc + tt + ttt);
        TabIter* dit = reinterpret_cast<TabIter*>(db + tp + tc + tt + ttt + tbs);
        static thread_local SingleArgs a;
        size_t cam_off = 0;
        int tile_off = 0, tab_tiles = 0, tab_blocks = 0;
        for (int i = 0; i < n; ++i) {
            fr_job* j = order[i];
            fr_volume v = job_volume(j, s->dtype);
            fill_problem(&v, j->cams.data(), j->d.ncam, &s->p, a);
            ProbDev& P = a.p;
            P.cams = dc + cam_off;
            P.targets = j->targets;
            P.bbox = j->bbox;
            P.residual = j->tabled ? nullptr : j->residual;
            P.partials = j->partials;
            P.dV = j->dV;
            P.img_in = j->residual;
            P.img_scale = 1.0f;
            P.list = j->flist;
            P.list_count = j->fbuf + flame_list_total_at(j->ntiles);
            P.vol_rw = j->vol;
            P.nodes = (long long)j->d.nx * j->d.ny * j->d.nz;
            P.sqerr = j->sqerr;
            P.ntiles = j->ntiles;
            P.iteration = j->iters_done;
            P.sq_slot = j->iters_done;
            if (j->d.alpha_l != 0.0f) P.alpha_l = j->d.alpha_l;
            P.pairs = j->pairs;
            P.tpart = j->tpart;
            P.nbx = bricks_along(j->d.nx);
            P.nby = bricks_along(j->d.ny);
            P.nbz = bricks_along(j->d.nz);
            P.occ = j->occ;
            P.occ_box = j->occ ? brick_box(j->occ, P.nbx, P.nby, P.nbz) : nullptr;
            P.hull = j->tags;
            P.hull_full = j->d.ncam >= 32 ? 0xffffffffu : ((1u << j->d.ncam) - 1u);
            P.adj_occ = j->hull_bricks;
            P.adj_box = j->hull_bricks ? brick_box(j->hull_bricks, P.nbx, P.nby, P.nbz) : nullptr;
            P.split_box = FR_SPLIT_BOX && kServerParts > 1 && j->hull_bricks && !(P.tau > 0.0f) ? 1 : 0;
            hp[i] = P;
            for (int k = 0; k < j->d.ncam; ++k) hc[cam_off + k] = a.cams[k];
            if (i < ntab) {
                htt[i] = tab_tiles;
                hbs[i] = tab_blocks;
                hit[i] = j->tab;
                tab_tiles += j->ntiles;
                tab_blocks += (int)tab_adjust_blocks(j->tab.nhull);
            } else {
                ht[i - ntab] = tile_off;
                tile_off += j->ntiles;
            }
            cam_off += (size_t)j->d.ncam;
        }
        ht[nm] = tile_off;
        htt[ntab] = tab_tiles;
        hbs[ntab] = tab_blocks;
        FR_CUDA(c, cudaMemcpyAsync(db, hb, tables, cudaMemcpyHostToDevice, st));
        FR_CUDA(c, cudaEventRecord(s->staging_done, st));
        const bool tau = s->p.tau > 0.0f;
        const bool hull = server_hull(s), skip = server_skip(s);
        ProbDev* dpm = dp + ntab;   // the marching jobs
        if (nm > 0) {
            if (skip) FR_CUDA(c, launch_brick_reset_batch(dpm, nm, st));
            FR_CUDA(c, launch_pair_pack_batch(dpm, nm, s->dtype, st));
            if (skip) FR_CUDA(c, launch_brick_box_batch(dpm, nm, st));
            FR_CUDA(c, launch_fwd_batch(dpm, dtl, nm, tile_off, s->dtype, KIND_RGB, tau, true, st, skip));
        }
        if (ntab > 0) FR_CUDA(c, launch_tab_forward_batch(dp, dit, dtt, ntab, tab_tiles, s->dtype, st));
        FR_CUDA(c, launch_finalize_batch(dp, n, 0, st));
        if (nm > 0) {
            FR_CUDA(c, launch_adjust_list_batch(dpm, dtl, nm, tile_off, s->dtype, tau, 0, st, hull && skip,
                                                kServerParts));
            FR_CUDA(c, launch_apply_batch(dpm, nm, s->dtype, s->p.clamp_nonneg, st));   // with the hull clear
        }
        if (ntab > 0)
            FR_CUDA(c, launch_tab_adjust_batch(dp, dit, dbs, ntab, tab_blocks, s->dtype, s->p.clamp_nonneg, st));
        FR_CUDA(c, cudaStreamSynchronize(st));
        // advance and retire
        for (size_t i = 0; i < s->resident.size();) {
            fr_job* j = s->resident[i];
            j->iters_done += 1;
            if (j->iters_done >= j->d.iters) {
                FR_TRY(job_complete(s, j));
                s->resident.erase(s->resident.begin() + i);
            } else {
                ++i;
            }
        }
    }
    if (running) *running = (int)s->resident.size();
    if (queued) *queued = (int)s->queue.size();
    return FR_OK;
}

extern "C" fr_status fr_job_get_info(const fr_job* j, fr_job_info* info)
{
    if (!j || !info) return FR_EINVAL;
    info->state = j->state;
    info->iters_done = j->iters_done;
    info->t_submit = j->t_submit;
    info->t_admit = j->t_admit;
    info->t_done = j->t_done;
    info->footprint = j->footprint;
    return FR_OK;
}

extern "C" fr_status fr_job_wait(fr_server* s, fr_job* j, int timeout_ms)
{
    if (!s || !j) return FR_EINVAL;
    const auto t_end = std::chrono::steady_clock::now() + std::chrono::milliseconds(timeout_ms);
    while (j->state == FR_JOB_QUEUED || j->state == FR_JOB_RUNNING) {
        if (std::chrono::steady_clock::now() > t_end) return FR_ETIMEDOUT;
        FR_TRY(fr_server_step(s, nullptr, nullptr));
    }
    return j->state == FR_JOB_DONE ? FR_OK : FR_ECANCELED;
}

extern "C" fr_status fr_job_cancel(fr_server* s, fr_job* j)
{
    if (!s || !j) return FR_EINVAL;
    if (j->state == FR_JOB_QUEUED || j->state == FR_JOB_RUNNING) j->cancel = true;
    return FR_OK;
}

extern "C" fr_status fr_job_release(fr_server* s, fr_job* j)
{
    if (!s || !j) return FR_EINVAL;
    if (j->state == FR_JOB_QUEUED || j->state == FR_JOB_RUNNING) return FR_EBUSY;
    delete j;
    return FR_OK;
}

extern "C" fr_status fr_server_memory(const fr_server* s, size_t* used, size_t* budget)
{
    if (!s) return FR_EINVAL;
    if (used) *used = s->used;
    if (budget) *budget = s->budget;
    return FR_OK;
}
