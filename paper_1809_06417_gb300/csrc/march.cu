// march.cu -- the ray-marching kernels of the reconstruction loop.
//
//  * fwd: renders every pixel (Eqs. 5-8; Algorithm 2, rendering half) and, in
//    the same pass, forms the residual of the colour constraint (Sec. 3.3.2)
//    and the squared-error partials of the error measure (Sec. 5.1).
//  * adjust: the paper's adjustment (Eqs. 10-12; Algorithm 2, adjustment half),
//    one thread per flame ray, accumulated with vector float reductions.
//  * backward: the exact gradient of the rendered images with the per-segment
//    transmittance recomputed along each ray.
//  * count: samples per render / per adjustment (for throughput accounting).
//
// One thread marches one ray; a CTA covers a 16 x 8 pixel tile of one view.
#include "fr_device.cuh"
#include "fr_internal.h"

// Launch bounds of the march kernels.  Building with -DFR_MARCH_MINB=n asks
// the compiler for n resident CTAs per SM (capping registers).
#ifdef FR_MARCH_MINB
#define FR_MARCH_BOUNDS __launch_bounds__(frk::kTileThreads, FR_MARCH_MINB)
#else
#define FR_MARCH_BOUNDS __launch_bounds__(frk::kTileThreads)
#endif
// Resident CTAs per SM asked for the forward march: 6 caps it at 80
// registers without spills (20% more warps than the 96 it takes unbounded;
// measured 3% faster).  The FP32 RGB field march with x-pair records and
// skipping (the reconstruction loop's) takes 7 (72 registers, 8 bytes
// spilled; 1% faster than 6 with the packed-pair blend); 8 spills 72 bytes.
#ifndef FR_FWD_MINB
#define FR_FWD_MINB 6
#endif
#ifndef FR_FWD_MINB_LOOP
#define FR_FWD_MINB_LOOP 7
#endif
#define FR_FWD_BOUNDS __launch_bounds__(frk::kTileThreads, FR_FWD_MINB)
#define FR_FWD_BOUNDS_T(DT, KIND, TAU, MODE) \
    __launch_bounds__(frk::kTileThreads, (DT) == DT_F32 && (KIND) == KIND_RGB && !(TAU) && (MODE) == 2 \
                                             ? FR_FWD_MINB_LOOP : FR_FWD_MINB)
// The adjustment over the flame-ray list runs one warp per CTA: a CTA's
// resources return as soon as its 32 rays end, where a 4-warp CTA waits for
// its longest ray (measured 6% faster).  FR_ADJ_MINB resident CTAs per SM
// leave the compiler 96 registers (20 warps per SM); 28 (72 registers)
// measured 2% slower.  The FP32 field adjustment with skipping (the
// reconstruction loop's) takes 24 (80 registers, no spill; 1% faster with
// the packed-pair weights), the others, which would spill there, 20.
#ifndef FR_ADJ_THREADS
#define FR_ADJ_THREADS 32
#endif
#ifndef FR_ADJ_MINB
#define FR_ADJ_MINB 20
#endif
#ifndef FR_ADJ_MINB_LOOP
#define FR_ADJ_MINB_LOOP 24
#endif
// The batched FP32 adjustment: 24 (80 registers, 68 bytes spilled) measured
// 2.8% faster on the video batch than 20 (219.0 against 213.0 frames/s); the
// 16-bit ones, which spill more there, keep FR_ADJ_MINB.
#ifndef FR_ADJ_BATCH_MINB
#define FR_ADJ_BATCH_MINB 24
#endif
#define FR_ADJ_LIST_BOUNDS __launch_bounds__(FR_ADJ_THREADS, FR_ADJ_MINB)
#define FR_ADJ_LIST_BOUNDS_T(DT, TAU, SKIP) \
    __launch_bounds__(FR_ADJ_THREADS, (DT) == DT_F32 && !(TAU) && (SKIP) ? FR_ADJ_MINB_LOOP : FR_ADJ_MINB)


namespace frk {

// ---------------------------------------------------------------------------
// Shared pieces
// ---------------------------------------------------------------------------

template <int DT, int KIND>
struct RecOf;
template <int DT>
struct RecOf<DT, KIND_RGB> {
    using T = float4;
    static __device__ __forceinline__ float4 load(const void* vol, long long i) { return load_rgb<DT>(vol, i); }
    static __device__ __forceinline__ void pair(const void* p, long long i, float4& a, float4& b)
    {
        load_rgb_pair<DT>(p, i, a, b);
    }
};
template <int DT>
struct RecOf<DT, KIND_TEMP> {
    using T = float2;
    static __device__ __forceinline__ float2 load(const void* vol, long long i) { return load_ts<DT>(vol, i); }
    static __device__ __forceinline__ void pair(const void* p, long long i, float2& a, float2& b)
    {
        load_ts_pair<DT>(p, i, a, b);
    }
};

// Source and extinction of a blended record (temperature through the table).
template <int KIND>
__device__ __forceinline__ void record_source(const ProbDev& P, float4 r, float S[3], float& sig, float dq[3])
{
    S[0] = r.x; S[1] = r.y; S[2] = r.z; sig = r.w;
}

__device__ __forceinline__ void record_source_temp(const ProbDev& P, float2 r, float S[3], float& sig, float dq[3])
{
    lut_eval(P, r.x, S, dq);
    sig = r.y;
}

// ---------------------------------------------------------------------------
// Forward render + residual
// ---------------------------------------------------------------------------

// The eight records of a cell, corner b = dx + 2 dy + 4 dz.
template <int DT, int KIND>
__device__ __forceinline__ void load8(const void* vol, long long base, int nx, long long nxy,
                                      typename RecOf<DT, KIND>::T v[8])
{
    using Rec = RecOf<DT, KIND>;
    v[0] = Rec::load(vol, base);
    v[1] = Rec::load(vol, base + 1);
    v[2] = Rec::load(vol, base + nx);
    v[3] = Rec::load(vol, base + nx + 1);
    v[4] = Rec::load(vol, base + nxy);
    v[5] = Rec::load(vol, base + nxy + 1);
    v[6] = Rec::load(vol, base + nxy + nx);
    v[7] = Rec::load(vol, base + nxy + nx + 1);
}

// The same from x-pair records: corners (0, dy, dz) and (1, dy, dz) in one load.
template <int DT, int KIND>
__device__ __forceinline__ void load8_pairs(const void* pairs, long long base, int nx, long long nxy,
                                            typename RecOf<DT, KIND>::T v[8])
{
    using Rec = RecOf<DT, KIND>;
    Rec::pair(pairs, base, v[0], v[1]);
    Rec::pair(pairs, base + nx, v[2], v[3]);
    Rec::pair(pairs, base + nxy, v[4], v[5]);
    Rec::pair(pairs, base + nxy + nx, v[6], v[7]);
}

// Staged forward gathers (FR_FWD_STAGE = 1, a comparison variant of the
// FP32 x-pair path): the next sample's cell records are copied asynchronously
// (cp.async) into the thread's own shared-memory slot one sample ahead, so the
// global load latency overlaps the current sample's arithmetic without a
// second set of records in registers.
#ifndef FR_FWD_STAGE
#define FR_FWD_STAGE 0
#endif

__device__ __forceinline__ void cp_async16(void* smem, const void* gmem)
{
    const unsigned s = (unsigned)__cvta_generic_to_shared(smem);
    asm volatile("cp.async.ca.shared.global [%0], [%1], 16;" :: "r"(s), "l"(gmem) : "memory");
}

__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }

__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_group 0;" ::: "memory"); }

// The four x-pair records of the cell at `base` into this thread's slot
// (stage[q][thread], q = 2 pair + half), as one cp.async group.
__device__ __forceinline__ void stage_cell(const void* pairs, long long base, int nx, long long nxy,
                                           float4 (*stage)[kTileThreads])
{
    const float* p = reinterpret_cast<const float*>(pairs);
    const long long idx[4] = {base, base + nx, base + nxy, base + nxy + nx};
#pragma unroll
    for (int q = 0; q < 4; ++q) {
        cp_async16(&stage[2 * q][threadIdx.x], p + 8 * idx[q]);
        cp_async16(&stage[2 * q + 1][threadIdx.x], p + 8 * idx[q] + 4);
    }
    cp_async_commit();
}

// Forward march of one ray.  Consecutive samples often share a cell (at half a
// voxel step about 2 in 5 do), so the cell's eight records stay in registers
// and are reloaded only when the sample enters another cell.  (Reloading just
// the four records of a crossed face costs more instructions than the L1
// traffic it saves; prefetching the next sample's cell into L1 measured 8%
// slower; one-warp CTAs, the tile's epilogue done by its last warp, 19% slower:
// a tile's four warps no longer share an SM's L1.)
// MODE 0: records gathered one by one; 1: from x-pair records; 2: x-pair
// records and exact skipping of empty bricks (RGB field mode only: a sample
// whose eight corner records are all zero adds exactly nothing and leaves the
// transmittance unchanged, so skipping it does not change the result).
// SPLIT: track the transmittance at the ray's part boundaries for a flame list
// of ray parts (the single-problem forward; the batched one lists no rays).
// One ray's results that a fused adjustment needs (fused_single).
struct FwdOut {
    bool flame;
    unsigned pix;
    float dl[3];   // residual of the colour constraint
    float tm;      // transmittance at the start of the ray's second part
};

template <int DT, int KIND, bool TAU, int MODE, bool SPLIT = false>
__device__ __forceinline__ void fwd_body(const ProbDev& P, const CamDev* cams, int tile, FwdOut* out = nullptr)
{
    constexpr bool PAIRS = MODE >= 1;
    constexpr bool SKIP = MODE == 2 && KIND == KIND_RGB && !TAU;
    using RT = typename RecOf<DT, KIND>::T;
    int view, px, py;
    tile_pixel(P, tile, view, px, py);
    const bool valid = px < P.W && py < P.H;
    float L0 = 0.0f, L1 = 0.0f, L2 = 0.0f;
    // transmittance after the samples of the ray's first j + 1 parts
    constexpr int kTm = SPLIT && FR_ADJ_SPLIT > 1 ? FR_ADJ_SPLIT - 1 : 1;
    float Tm[kTm];
#pragma unroll
    for (int j = 0; j < kTm; ++j) Tm[j] = 1.0f;
    if (valid) {
        Ray R;
        if (make_ray(cams[view], px, py, P.nx, P.ny, P.nz, P.step, R)) {
            const long long nxy = (long long)P.nx * P.ny;
            RT v[8];
#pragma unroll
            for (int q = 0; q < 8; ++q) v[q] = RT{};
            long long vbase = -1;
#if FR_FWD_STAGE
            long long staged = -1;   // the cell whose records are in flight to (or in) the thread's slot
#endif
            float T = 1.0f;
            BrickSkip skip;
            int k0 = 0, k1 = R.n;
            if constexpr (SKIP) {
                if (!BrickSkip::box_range(P, P.occ_box, R, P.step, k0, k1)) k1 = 0;
            }
            int kb[kTm];
            if constexpr (SPLIT && FR_ADJ_SPLIT > 1) {
                // the part boundaries the adjustment uses: its box range
                // (P.split_box, the adjustment's own box_range over adj_box),
                // else the whole chord
                int sa = 0, sn = R.n;
                if (SKIP && P.split_box && P.occ_box == P.adj_box) {
                    // the march clips to that box itself: its own range
                    sa = k0;
                    sn = max(k1 - k0, 0);
                } else if (P.split_box) {
                    int a0 = 0, a1 = R.n;
                    const bool any = BrickSkip::box_range(P, P.adj_box, R, P.step, a0, a1);
                    sa = any ? a0 : 0;
                    sn = any ? a1 - a0 : 0;
                }
#pragma unroll
                for (int j = 0; j < kTm; ++j) kb[j] = sa + sn * (j + 1) / FR_ADJ_SPLIT;
            }
            for (int k = k0; k < k1; ++k) {
                float len, x, y, z;
                segment(R, P.step, k, len, x, y, z);
                if constexpr (SKIP) {
                    if (skip.empty(P.occ, P, R, P.step, x, y, z, k)) continue;
                }
                const Cell c = cell_of(x, y, z, P.nx, P.ny, P.nz);
                if constexpr (PAIRS && KIND == KIND_RGB && DT == DT_F32) {
#if FR_FWD_STAGE
                    __shared__ float4 stage[8][kTileThreads];
                    const long long lim = nxy * P.nz - nxy - P.nx - 1;   // largest cell base
                    (void)lim;
                    if (c.base != vbase) {
                        // the staged cell, or (after a skip) this one, staged now
                        if (staged != c.base) {
                            cp_async_wait_all();
                            stage_cell(P.pairs, FR_CHK(c.base, lim, 1u), P.nx, nxy, stage);
                        }
                        cp_async_wait_all();
#pragma unroll
                        for (int q = 0; q < 8; ++q) v[q] = stage[q][threadIdx.x];
                        staged = -1;
                        vbase = c.base;
                    }
                    // the next sample's cell, one sample ahead
                    if (k + 1 < k1 && staged < 0) {
                        float l2, x2, y2, z2;
                        segment(R, P.step, k + 1, l2, x2, y2, z2);
                        const long long nb = cell_of(x2, y2, z2, P.nx, P.ny, P.nz).base;
                        if (nb != vbase) {
                            stage_cell(P.pairs, FR_CHK(nb, lim, 1u), P.nx, nxy, stage);
                            staged = nb;
                        }
                    }
#else
                    // The four pair loads predicated on a cell change rather
                    // than branched on it: the lanes, which enter cells at
                    // different samples, stay converged (2.4% faster).
                    const unsigned need = c.base != vbase ? 1u : 0u;
                    vbase = c.base;
                    // the cell's far corner, base + nxy + nx + 1, must be a node
                    const long long b = FR_CHK(c.base, nxy * P.nz - nxy - P.nx - 1, 1u);
                    const long long idx[4] = {b, b + P.nx, b + nxy, b + nxy + P.nx};
#pragma unroll
                    for (int q = 0; q < 4; ++q) load_rgb_pair_f32_if(P.pairs, idx[q], need, v[2 * q], v[2 * q + 1]);
#endif
                } else
                if (c.base != vbase) {
                    vbase = c.base;
                    // the cell's far corner, base + nxy + nx + 1, must be a node
                    const long long b = FR_CHK(c.base, nxy * P.nz - nxy - P.nx - 1, 1u);
                    if constexpr (PAIRS) load8_pairs<DT, KIND>(P.pairs, b, P.nx, nxy, v);
                    else load8<DT, KIND>(P.vol, b, P.nx, nxy, v);
                }
                const RT r = slot_blend<RT>(v, c.fx, c.fy, c.fz);
                float S[3], sig, dq[3];
                if constexpr (KIND == KIND_RGB) record_source<KIND>(P, r, S, sig, dq);
                else record_source_temp(P, r, S, sig, dq);
                if constexpr (TAU) {
                    const float w = T * P.tau;
                    L0 = fmaf(w, S[0], L0); L1 = fmaf(w, S[1], L1); L2 = fmaf(w, S[2], L2);
                    T *= 1.0f - P.tau;
                } else {
                    const float e = __expf(-sig * len);
                    const float w = T * seg_weight(sig, len, e);
                    L0 = fmaf(w, S[0], L0); L1 = fmaf(w, S[1], L1); L2 = fmaf(w, S[2], L2);
                    T *= e;
                }
                if constexpr (SPLIT && FR_ADJ_SPLIT > 1) {
#pragma unroll
                    for (int j = 0; j < kTm; ++j) Tm[j] = k < kb[j] ? T : Tm[j];
                }
            }
#if FR_FWD_STAGE
            // a copy for a cell the ray did not reach lands before the thread moves on
            cp_async_wait_all();
#endif
        }
    }
    // pixel epilogue: image, residual of the colour constraint, error sums
    float a0 = 0.0f, a1 = 0.0f, a2 = 0.0f, cnt = 0.0f;
    float fl0 = 0.0f, fl1 = 0.0f, fl2 = 0.0f;   // the residual (kept for a fused adjustment)
    const long long pix = valid ? FR_CHK(((long long)view * P.H + py) * P.W + px, (long long)P.ncam * P.H * P.W, 4u)
                                : 0;
    bool flame = false;
    if (valid) {
        if (P.rendered) {
            float* o = P.rendered + 3 * pix;
            o[0] = L0; o[1] = L1; o[2] = L2;
        }
        if (P.targets) {
            const float* t = P.targets + 3 * pix;
            const float t0 = t[0], t1 = t[1], t2 = t[2];
            const float d0 = t0 - L0, d1 = t1 - L1, d2 = t2 - L2;
            flame = fmaxf(t0, fmaxf(t1, t2)) > P.thresh;
            if (P.residual) {
                float* r = P.residual + 3 * pix;
                r[0] = flame ? d0 : 0.0f;
                r[1] = flame ? d1 : 0.0f;
                r[2] = flame ? d2 : 0.0f;
            }
            fl0 = d0; fl1 = d1; fl2 = d2;
            const int* bb = P.bbox + 4 * view;
            if (px >= bb[0] && px <= bb[2] && py >= bb[1] && py <= bb[3]) {
                a0 = d0 * d0; a1 = d1 * d1; a2 = d2 * d2; cnt = 1.0f;
            }
        }
    }
    if (P.flist) {
        // flame-ray list for the adjustment: each CTA appends the flame
        // pixels of its tile as one contiguous run in tile order, padded to
        // whole warps, so each of the adjustment's warps takes neighbouring
        // rays of one tile (measured 3% faster than unpadded runs, whose
        // warps straddle two unrelated tiles).  With flist_tm the run holds
        // one such block per part of the rays, part j's entries tagged j in
        // their top two bits and carrying the transmittance Tm[j - 1].
        __shared__ unsigned wcount[kTileThreads / 32];
        __shared__ unsigned run_at, run_len;
        const unsigned m = __ballot_sync(0xffffffffu, flame);
        const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
        if (lane == 0) wcount[w] = (unsigned)__popc(m);
        __syncthreads();
        const unsigned parts = SPLIT && FR_ADJ_SPLIT > 1 && P.flist_tm ? (unsigned)FR_ADJ_SPLIT : 1u;
        if (threadIdx.x == 0) {
            unsigned total = 0;
#pragma unroll
            for (int i = 0; i < kTileThreads / 32; ++i) total += wcount[i];
            run_len = total;
            total = (total + 31u) & ~31u;
            run_at = total ? atomicAdd(P.flist_count, parts * total) : 0u;
        }
        __syncthreads();
        const unsigned padded = (run_len + 31u) & ~31u;
        if (flame) {
            unsigned at = run_at + (unsigned)__popc(m & ((1u << lane) - 1u));
            for (int i = 0; i < w; ++i) at += wcount[i];
            P.flist[at] = (unsigned)pix;
            if (P.flist_dl) {
                float* q = P.flist_dl + 3 * (size_t)at;
                q[0] = fl0; q[1] = fl1; q[2] = fl2;
            }
            if (parts > 1u) {
#pragma unroll
                for (int j = 1; j <= kTm; ++j) {
                    P.flist[at + j * padded] = (unsigned)pix | ((unsigned)j << 30);
                    P.flist_tm[at + j * padded] = Tm[j - 1];
                    if (P.flist_dl) {
                        float* q = P.flist_dl + 3 * (size_t)(at + j * padded);
                        q[0] = fl0; q[1] = fl1; q[2] = fl2;
                    }
                }
            }
        }
        // the run is padded to whole warps with entries that name no pixel
        if ((unsigned)threadIdx.x >= run_len && (unsigned)threadIdx.x < padded) {
            for (unsigned j = 0; j < parts; ++j) P.flist[run_at + j * padded + threadIdx.x] = kNoPixel;
        }
    }
    if constexpr (SPLIT && FR_ADJ_SPLIT > 1) {
        // batched problems: the transmittance at each part boundary of a
        // flame pixel, read by the adjustment of that part
        if (P.tpart && flame) {
            const long long npix = (long long)P.ncam * P.H * P.W;
#pragma unroll
            for (int j = 0; j < kTm; ++j) P.tpart[j * npix + pix] = Tm[j];
        }
    }
    if (P.partials) {
        __shared__ float red[4][kTileThreads / 32];
        a0 = warp_sum(a0); a1 = warp_sum(a1); a2 = warp_sum(a2); cnt = warp_sum(cnt);
        const int w = threadIdx.x >> 5;
        if ((threadIdx.x & 31) == 0) { red[0][w] = a0; red[1][w] = a1; red[2][w] = a2; red[3][w] = cnt; }
        __syncthreads();
        if (threadIdx.x < 4) {
            float s = 0.0f;
#pragma unroll
            for (int i = 0; i < kTileThreads / 32; ++i) s += red[threadIdx.x][i];
            P.partials[4 * (long long)tile + threadIdx.x] = s;
        }
    }
    if (out) {
        out->flame = flame;
        out->pix = (unsigned)pix;
        out->dl[0] = fl0; out->dl[1] = fl1; out->dl[2] = fl2;
        out->tm = Tm[0];
    }
}

template <int DT, int KIND, bool TAU, int MODE>
__global__ void FR_FWD_BOUNDS_T(DT, KIND, TAU, MODE) fwd_single(const __grid_constant__ SingleArgs a)
{
    const int tile = a.p.tile_order ? (int)__ldg(a.p.tile_order + blockIdx.x) : (int)blockIdx.x;
    fwd_body<DT, KIND, TAU, MODE, true>(a.p, a.cams, tile);
}

// Launch order of the forward's tiles, longest first: per tile, the most
// samples one of its rays takes inside the box (box_range over `box`, the
// whole chord without one) as a key, then a counting sort by decreasing key
// in one CTA (positions inside a key taken with atomics: any order).
constexpr int kOrderKeys = 1024;
__global__ void __launch_bounds__(kTileThreads) tile_work_kernel(const __grid_constant__ SingleArgs a,
                                                                 const unsigned* box, unsigned* key)
{
    const ProbDev& P = a.p;
    int view, px, py;
    tile_pixel(P, blockIdx.x, view, px, py);
    int n = 0;
    if (px < P.W && py < P.H) {
        Ray R;
        if (make_ray(a.cams[view], px, py, P.nx, P.ny, P.nz, P.step, R)) {
            int k0 = 0, k1 = R.n;
            if (!box || BrickSkip::box_range(P, box, R, P.step, k0, k1)) n = max(k1 - k0, 0);
            else n = 0;
        }
    }
    __shared__ int wm[kTileThreads / 32];
    n = __reduce_max_sync(0xffffffffu, n);
    if ((threadIdx.x & 31) == 0) wm[threadIdx.x >> 5] = n;
    __syncthreads();
    if (threadIdx.x == 0) {
        int m = 0;
        for (int i = 0; i < kTileThreads / 32; ++i) m = max(m, wm[i]);
        key[blockIdx.x] = (unsigned)min(m / 2, kOrderKeys - 1);
    }
}

__global__ void __launch_bounds__(1024) tile_order_kernel(const unsigned* __restrict__ key, int ntiles,
                                                          unsigned* __restrict__ order)
{
    __shared__ unsigned cnt[kOrderKeys];
    for (int i = threadIdx.x; i < kOrderKeys; i += 1024) cnt[i] = 0;
    __syncthreads();
    for (int t = threadIdx.x; t < ntiles; t += 1024) atomicAdd(&cnt[kOrderKeys - 1 - __ldg(key + t)], 1u);
    __syncthreads();
    if (threadIdx.x == 0) {
        unsigned run = 0;
        for (int i = 0; i < kOrderKeys; ++i) {
            const unsigned c = cnt[i];
            cnt[i] = run;
            run += c;
        }
    }
    __syncthreads();
    for (int t = threadIdx.x; t < ntiles; t += 1024) {
        const unsigned at = atomicAdd(&cnt[kOrderKeys - 1 - __ldg(key + t)], 1u);
        order[at] = (unsigned)t;
    }
}

// (Batched forward: capped at 80 registers (6 CTAs per SM) it spills and is
// still 3% faster on the video batch than with 96 registers, and 1% faster
// than at 72 (7 CTAs, 136 bytes spilled); FR_FWD_BATCH_CAP=0 leaves the
// registers unbounded.)
#ifndef FR_FWD_BATCH_CAP
#define FR_FWD_BATCH_CAP 1
#endif
#ifndef FR_FWD_BATCH_MINB
#define FR_FWD_BATCH_MINB FR_FWD_MINB
#endif
#if FR_FWD_BATCH_CAP
#define FR_FWD_BATCH_BOUNDS __launch_bounds__(frk::kTileThreads, FR_FWD_BATCH_MINB)
#else
#define FR_FWD_BATCH_BOUNDS FR_MARCH_BOUNDS
#endif
// FR_BATCH_PARTS: parts each flame ray of a batch (and of the server) is
// adjusted in.  1 (whole rays): the split, which makes the single-problem
// adjustment 6% faster, measured 8% slower on the video batch (64 frames of
// 96^3, 8 views of 384^2) and 10% lower in serving capacity, where many short
// problems already fill the GPU's last wave and the forward's part bookkeeping
// spills.
#ifndef FR_BATCH_PARTS
#define FR_BATCH_PARTS 1
#endif
static_assert(FR_BATCH_PARTS == 1 || FR_BATCH_PARTS == FR_ADJ_SPLIT, "batched parts: 1 or FR_ADJ_SPLIT");
template <int DT, int KIND, bool TAU, int MODE>
__global__ void FR_FWD_BATCH_BOUNDS fwd_batch(const ProbDev* __restrict__ probs, const int* __restrict__ tile_start,
                                              int nprob)
{
    const int p = find_problem(tile_start, nprob, blockIdx.x);
    const ProbDev& P = probs[p];
    fwd_body<DT, KIND, TAU, MODE, (FR_BATCH_PARTS > 1)>(P, P.cams, blockIdx.x - __ldg(tile_start + p));
}

// ---------------------------------------------------------------------------
// Adjustment, paper rule (Eqs. 10-12)
// ---------------------------------------------------------------------------

// dL is constant along a ray, so each key point collects the scalar sum of
// G alpha_l T exp(-alpha_d D) over the ray's samples in its window slot and
// receives that sum times dL when the ray leaves it.
// RG: G(s) drawn per sample (g_std > 0); false: G = 1 (a compile-time
// constant, 1.6% faster than a per-sample test of g_std).
// Accumulator of the key points' sums a ray releases, for the comparison of
// FR_ADJ_ACCUM = 1 (see adj_list_tab): an open-addressing table of one CTA's
// key points in shared memory, flushed with vector reductions when the CTA's
// rays are done.
#ifndef FR_ADJ_TAB_BITS
#define FR_ADJ_TAB_BITS 10
#endif
constexpr int kTab = 1 << FR_ADJ_TAB_BITS;
struct KeyTable {
    int key[kTab];           // node index, -1 while free
    float v[kTab][3];
};

// Adds {a, b, c} to node's entry (claimed with a compare-and-swap on its
// first visit); after 8 occupied probes the sum goes straight to dV.
__device__ __forceinline__ void tab_add(KeyTable& T, unsigned node, float a, float b, float c, float* dV)
{
    unsigned h = (node * 2654435761u) >> (32 - FR_ADJ_TAB_BITS);
    const volatile int* keys = T.key;
#pragma unroll 1
    for (int probe = 0; probe < 8; ++probe) {
        int k = keys[h];
        if (k == -1) k = atomicCAS(&T.key[h], -1, (int)node);
        if (k == -1 || k == (int)node) {
            atomicAdd(&T.v[h][0], a);
            atomicAdd(&T.v[h][1], b);
            atomicAdd(&T.v[h][2], c);
            return;
        }
        h = (h + 1) & (kTab - 1);
    }
    red_add_v4(dV + 4 * (size_t)node, a, b, c, 0.0f);
}

template <int DT, bool TAU, bool SKIP, bool RG, int ACC = 0>
__device__ __forceinline__ void adj_ray(const ProbDev& P, const CamDev* cams, int view, int px, int py,
                                        int iteration, int part = -1, float T0 = 1.0f, KeyTable* tab = nullptr,
                                        const float* dl_in = nullptr)
{
    // SKIP: samples in bricks with no key point inside the visual hull are
    // skipped.  Their records are zero (no extinction: T is unchanged) and
    // their key points' updates are discarded after the update, so the
    // result is the same.  dl_in (nullable): the ray's residual, else read
    // from P.img_in.
    const long long pix = ((long long)view * P.H + py) * P.W + px;
    const float* g = dl_in ? dl_in : P.img_in + 3 * pix;
    const float sc = dl_in ? 1.0f : P.img_scale;
    const float dl0 = g[0] * sc, dl1 = g[1] * sc, dl2 = g[2] * sc;
    if (dl0 == 0.0f && dl1 == 0.0f && dl2 == 0.0f) return;
    Ray R;
    if (!make_ray(cams[view], px, py, P.nx, P.ny, P.nz, P.step, R)) return;
    const long long nxy = (long long)P.nx * P.ny;
    const int nxy32 = P.nx * P.ny;
    const int pixel = py * P.W + px;
    const float dcoef = -P.alpha_d * kLog2e;
    float acc[8], sg[8];
#pragma unroll
    for (int t = 0; t < 8; ++t) { acc[t] = 0.0f; sg[t] = 0.0f; }
    float* dV = P.dV;
    const void* vol = P.vol;
    const long long nodes = nxy * P.nz;
    (void)nodes;
    // The window's callbacks run for every slot at every sample with p telling
    // whether the slot moves, and predicate their memory operations on it: no
    // branch, so the warp's lanes, which change cells at different samples,
    // stay converged (2.6% faster than branching per slot).  Every slot that
    // leaves has collected at least one sample, so its reduction is issued
    // without testing the weight (a zero test per slot measured 5% slower).
    // (Reloading all eight corner sigmas on every cell change instead of the
    // entering slots' measured 16% slower.)
    auto leave = [&acc, dV, dl0, dl1, dl2, nodes, tab](int t, int node, bool p) {
        const float w = acc[t];
        if constexpr (ACC == 0) {
            red_add_v4_if(dV + 4 * (unsigned)FR_CHK(node, nodes, 2u), w * dl0, w * dl1, w * dl2, 0.0f, p);
        } else {
            if (p) tab_add(*tab, (unsigned)FR_CHK(node, nodes, 2u), w * dl0, w * dl1, w * dl2, dV);
        }
        acc[t] = p ? 0.0f : w;
    };
    auto enter = [&sg, vol, nodes](int t, int node, bool p) {
        if constexpr (!TAU) {
            // sigma is the record's fourth component (16-bit records widened
            // in the predicated load too: a branch per slot for them measured
            // 6% slower; a packed FP32 sigma array written by the pack, for
            // denser L1 lines, measured the same within 1%)
            const long long at = 4 * (long long)(unsigned)FR_CHK(node, nodes, 1u) + 3;
            if constexpr (DT == DT_F32) load_f32_if(reinterpret_cast<const float*>(vol) + at, p, sg[t]);
            else if constexpr (DT == DT_BF16) load_bf16_if(reinterpret_cast<const unsigned short*>(vol) + at, p, sg[t]);
            else load_f16_if(reinterpret_cast<const unsigned short*>(vol) + at, p, sg[t]);
        }
    };
    Win W;
    W.live = false;
    float T = T0;
    BrickSkip skip;
    int k0 = 0, k1 = R.n;
    if constexpr (SKIP) {
        if (!BrickSkip::box_range(P, P.adj_box, R, P.step, k0, k1)) return;
    }
#if FR_ADJ_SPLIT > 1
    // part j: samples [a + m j / n, a + m (j + 1) / n) of the ray -- [a, a + m)
    // the box range (P.split_box), else the whole chord [0, R.n) -- starting
    // from the transmittance the forward march reached there
    if (part >= 0) {
        const bool in_box = SKIP && P.split_box;
        const int sa = in_box ? k0 : 0, sn = in_box ? k1 - k0 : R.n;
        const int a0 = sa + sn * part / FR_ADJ_SPLIT, a1 = sa + sn * (part + 1) / FR_ADJ_SPLIT;
        k0 = max(k0, a0);
        k1 = min(k1, a1);
    }
#endif
    for (int k = k0; k < k1; ++k) {
        float len, x, y, z;
        segment(R, P.step, k, len, x, y, z);
        const CellIJK c = cell_ijk(x, y, z, P.nx, P.ny, P.nz);
        // (testing the brick only when the cell changes measured 5% slower)
        if constexpr (SKIP) {
            if (skip.empty_at(P.adj_occ, P, R, P.step, c, k)) continue;
        }
        win_move_pred(W, c.i, c.j, c.k, P.nx, P.ny, nxy32, leave, enter);
        const float gx = mirror_frac(c.i, c.fx), gy = mirror_frac(c.j, c.fy), gz = mirror_frac(c.k, c.fz);
        float G = 1.0f;
        if constexpr (RG) G = g_draw(P.seed, P.g_std, iteration, view + P.view_base, pixel, k);
        const float base = G * P.alpha_l * T;
        // squared distances (voxel units) from the sample to each slot's key point
        const float ex[2] = {gx * gx, (1.0f - gx) * (1.0f - gx)};
        const float ey[2] = {gy * gy, (1.0f - gy) * (1.0f - gy)};
        const float ez[2] = {gz * gz, (1.0f - gz) * (1.0f - gz)};
        const float exy[4] = {ex[0] + ey[0], ex[1] + ey[0], ex[0] + ey[1], ex[1] + ey[1]};
#if FR_PACKED
        // slots t and t + 4 side by side (the same operations per slot)
        const F2 ezz = f2(ez[0], ez[1]), bb = f2(base, base), cc = f2(dcoef, dcoef);
#pragma unroll
        for (int t = 0; t < 4; ++t) {
            const float2 d = f2_get(f2_add(f2(exy[t], exy[t]), ezz));
            float r0, r1;
            asm("sqrt.approx.ftz.f32 %0, %1;" : "=f"(r0) : "f"(d.x));
            asm("sqrt.approx.ftz.f32 %0, %1;" : "=f"(r1) : "f"(d.y));
            const float2 e = f2_get(f2_mul(cc, f2(r0, r1)));
            const float2 a2 = f2_get(f2_fma(bb, f2(ex2_approx(e.x), ex2_approx(e.y)), f2(acc[t], acc[t + 4])));
            acc[t] = a2.x;
            acc[t + 4] = a2.y;
        }
#else
#pragma unroll
        for (int t = 0; t < 8; ++t) acc[t] = fmaf(base, dist_weight(dcoef, exy[t & 3] + ez[t >> 2]), acc[t]);
#endif
        if constexpr (TAU) T *= 1.0f - P.tau;
        else T *= __expf(-slot_blend<float>(sg, gx, gy, gz) * len);
    }
    (void)nxy;
    win_release(W, [&leave](int t, int node) { leave(t, node, true); });
}

template <int DT, bool TAU>
__device__ __forceinline__ void adj_body(const ProbDev& P, const CamDev* cams, int tile)
{
    int view, px, py;
    tile_pixel(P, tile, view, px, py);
    if (px >= P.W || py >= P.H) return;
    if (P.g_std > 0.0f) adj_ray<DT, TAU, false, true>(P, cams, view, px, py, P.iteration);
    else adj_ray<DT, TAU, false, false>(P, cams, view, px, py, P.iteration);
}

// The same over a compacted list of flame rays (linear pixel indices in tile
// order, so a warp's 32 rays are neighbours): no lane idles on a non-flame
// pixel.  CTA b takes list entries [n b, n b + n), n = FR_ADJ_THREADS.  With
// tm, an entry names one part of a ray (its top two bits) and the part starts
// from the transmittance tm holds at the entry's position; the parts'
// contributions add up to the whole ray's, the key points at a part boundary
// receiving one reduction from each side.
// (A persistent grid whose warps take the list's 32-entry runs from a
// segment owned by their SM, so that one SM marches neighbouring rays and
// shares their records in L1, stealing from the fullest segment at the end,
// measured 9% slower: the GPU then works on one region per SM at once
// instead of one contiguous stretch of the list.  The same grid taking the
// runs in list order from one global counter measured 6% slower: the CTAs
// past the list's end, which exit at once, cost less than a warp's wait for
// its next chunk.)
template <int DT, bool TAU, bool SKIP>
__global__ void FR_ADJ_LIST_BOUNDS_T(DT, TAU, SKIP) adj_list(const __grid_constant__ SingleArgs a,
                                                          const unsigned* __restrict__ list,
                                         const unsigned* __restrict__ count, const float* __restrict__ tm)
{
    const unsigned i = blockIdx.x * (unsigned)FR_ADJ_THREADS + threadIdx.x;
    if (i >= __ldg(count)) return;
    const ProbDev& P = a.p;
    unsigned e = __ldg(list + i);
    if (e == kNoPixel) return;
    int part = -1;
    float T0 = 1.0f;
    if (tm) {
        part = (int)(e >> 30);
        e &= 0x3fffffffu;
        if (part) T0 = __ldg(tm + i);
    }
    const unsigned pix = (unsigned)FR_CHK(e, (long long)P.ncam * P.W * P.H, 8u);
    const unsigned per_view = (unsigned)P.W * (unsigned)P.H;
    const int view = (int)(pix / per_view);
    const unsigned r = pix - (unsigned)view * per_view;
    const int py = (int)(r / (unsigned)P.W), px = (int)(r - (unsigned)py * (unsigned)P.W);
    const int it = P.iteration + (P.iter_dev ? __ldg(P.iter_dev) : 0);
    const float* dl = P.flist_dl ? P.flist_dl + 3 * (size_t)i : nullptr;
    if (P.g_std > 0.0f) adj_ray<DT, TAU, SKIP, true>(P, a.cams, view, px, py, it, part, T0, nullptr, dl);
    else adj_ray<DT, TAU, SKIP, false>(P, a.cams, view, px, py, it, part, T0, nullptr, dl);
}

// Forward march and paper-rule adjustment of one tile in one kernel
// (FR_FUSED = 1, a comparison variant of the loop's fwd_single + adj_list):
// the tile's rays march forward (fwd_body: image sums, error partials), its
// flame pixels' index, residual and transmittance at the ray's middle sample
// go to shared memory instead of a flame-ray list in global memory, and the
// CTA's warps then adjust those rays in FR_ADJ_SPLIT parts while the records
// they gathered are still in the SM's L1.  No residual image is written.
#ifndef FR_FUSED
#define FR_FUSED 0
#endif
#ifndef FR_FUSED_MINB
#define FR_FUSED_MINB 5
#endif
#if FR_FUSED
template <int DT, bool SKIP_ADJ>
__global__ void __launch_bounds__(kTileThreads, FR_FUSED_MINB) fused_single(const __grid_constant__ SingleArgs a)
{
    static_assert(FR_ADJ_SPLIT <= 2, "the fused form keeps one part boundary per ray");
    FwdOut o;
    fwd_body<DT, KIND_RGB, false, 2, true>(a.p, a.cams, blockIdx.x, &o);
    __shared__ unsigned f_pix[kTileThreads];
    __shared__ float f_dl[3][kTileThreads];
    __shared__ float f_tm[kTileThreads];
    __shared__ unsigned f_wc[kTileThreads / 32];
    const unsigned m = __ballot_sync(0xffffffffu, o.flame);
    const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (lane == 0) f_wc[w] = (unsigned)__popc(m);
    __syncthreads();
    unsigned at = (unsigned)__popc(m & ((1u << lane) - 1u)), F = 0;
#pragma unroll
    for (int i = 0; i < kTileThreads / 32; ++i) {
        if (i < w) at += f_wc[i];
        F += f_wc[i];
    }
    if (o.flame) {
        f_pix[at] = o.pix;
        f_dl[0][at] = o.dl[0];
        f_dl[1][at] = o.dl[1];
        f_dl[2][at] = o.dl[2];
        f_tm[at] = o.tm;
    }
    __syncthreads();
    const ProbDev& P = a.p;
    const unsigned parts = (unsigned)FR_ADJ_SPLIT, items = F * parts;
    const int it = P.iteration + (P.iter_dev ? __ldg(P.iter_dev) : 0);
    const unsigned per_view = (unsigned)P.W * (unsigned)P.H;
    for (unsigned item = threadIdx.x; item < items; item += kTileThreads) {
        const unsigned part = item / F, idx = item - part * F;
        const unsigned pix = f_pix[idx];
        const float dl[3] = {f_dl[0][idx], f_dl[1][idx], f_dl[2][idx]};
        const int view = (int)(pix / per_view);
        const unsigned r = pix - (unsigned)view * per_view;
        const int py = (int)(r / (unsigned)P.W), px = (int)(r - (unsigned)py * (unsigned)P.W);
        const int pp = parts > 1u ? (int)part : -1;
        const float T0 = part ? f_tm[idx] : 1.0f;
        if (P.g_std > 0.0f) adj_ray<DT, false, SKIP_ADJ, true>(P, a.cams, view, px, py, it, pp, T0, nullptr, dl);
        else adj_ray<DT, false, SKIP_ADJ, false>(P, a.cams, view, px, py, it, pp, T0, nullptr, dl);
    }
}
#endif

// adj_list with each CTA's key-point sums gathered in a shared-memory table
// (KeyTable) and flushed with one vector reduction per key point the CTA's
// rays touched, instead of one per key point a ray leaves (FR_ADJ_ACCUM = 1;
// a comparison variant, one warp per CTA).
#ifndef FR_ADJ_ACCUM
#define FR_ADJ_ACCUM 0
#endif
template <int DT, bool TAU, bool SKIP>
__global__ void FR_ADJ_LIST_BOUNDS adj_list_tab(const __grid_constant__ SingleArgs a,
                                                const unsigned* __restrict__ list,
                                                const unsigned* __restrict__ count, const float* __restrict__ tm)
{
    static_assert(FR_ADJ_THREADS == 32, "one warp per CTA");
    __shared__ KeyTable tab;
    const unsigned n = __ldg(count);
    const unsigned i = blockIdx.x * 32u + threadIdx.x;
    if (blockIdx.x * 32u >= n) return;                 // the whole CTA past the list's end
    for (int j = threadIdx.x; j < kTab; j += 32) {
        tab.key[j] = -1;
        tab.v[j][0] = tab.v[j][1] = tab.v[j][2] = 0.0f;
    }
    __syncwarp();
    const ProbDev& P = a.p;
    unsigned e = i < n ? __ldg(list + i) : kNoPixel;
    if (e != kNoPixel) {
        int part = -1;
        float T0 = 1.0f;
        if (tm) {
            part = (int)(e >> 30);
            e &= 0x3fffffffu;
            if (part) T0 = __ldg(tm + i);
        }
        const unsigned pix = (unsigned)FR_CHK(e, (long long)P.ncam * P.W * P.H, 8u);
        const unsigned per_view = (unsigned)P.W * (unsigned)P.H;
        const int view = (int)(pix / per_view);
        const unsigned r = pix - (unsigned)view * per_view;
        const int py = (int)(r / (unsigned)P.W), px = (int)(r - (unsigned)py * (unsigned)P.W);
        const int it = P.iteration + (P.iter_dev ? __ldg(P.iter_dev) : 0);
        const float* dl = P.flist_dl ? P.flist_dl + 3 * (size_t)i : nullptr;
        if (P.g_std > 0.0f) adj_ray<DT, TAU, SKIP, true, 1>(P, a.cams, view, px, py, it, part, T0, &tab, dl);
        else adj_ray<DT, TAU, SKIP, false, 1>(P, a.cams, view, px, py, it, part, T0, &tab, dl);
    }
    __syncwarp();
    for (int j = threadIdx.x; j < kTab; j += 32) {
        const int k = tab.key[j];
        if (k >= 0) red_add_v4(P.dV + 4 * (size_t)k, tab.v[j][0], tab.v[j][1], tab.v[j][2], 0.0f);
    }
}

// Batched form, one warp per CTA like adj_list: CTA b covers list entries
// [n b', n b' + n) of the problem whose tile range holds tile
// b / (parts 128 / n), b' counted from that problem's first CTA
// (n = FR_ADJ_THREADS).  With parts > 1 every problem's list holds `parts`
// entries per flame ray (ProbDev::tpart), part j starting from the
// transmittance the forward stored for it.  The G(s) stream index is the
// problem's own iteration plus `iteration`.
template <int DT, bool TAU, bool SKIP>
__global__ void __launch_bounds__(FR_ADJ_THREADS, (DT) == DT_F32 ? FR_ADJ_BATCH_MINB : FR_ADJ_MINB) adj_list_batch(const ProbDev* __restrict__ probs,
                                                  const int* __restrict__ tile_start, int nprob, int iteration,
                                                  unsigned parts)
{
    const unsigned per = parts * (unsigned)(kTileThreads / FR_ADJ_THREADS);   // CTAs per tile
    const int p = find_problem(tile_start, nprob, (int)(blockIdx.x / per));
    const ProbDev& P = probs[p];
    const unsigned i = (blockIdx.x - (unsigned)__ldg(tile_start + p) * per) * (unsigned)FR_ADJ_THREADS + threadIdx.x;
    if (i >= __ldg(P.list_count)) return;
    unsigned e = __ldg(P.list + i);
    if (e == kNoPixel) return;
    int part = -1;
    float T0 = 1.0f;
    if (parts > 1u) {
        part = (int)(e >> 30);
        e &= 0x3fffffffu;
    }
    const unsigned per_view = (unsigned)P.W * (unsigned)P.H;
    const unsigned pix = (unsigned)FR_CHK(e, (long long)P.ncam * per_view, 8u);
    if (part > 0) T0 = __ldg(P.tpart + (size_t)(part - 1) * P.ncam * per_view + pix);
    const int view = (int)(pix / per_view);
    const unsigned r = pix - (unsigned)view * per_view;
    const int py = (int)(r / (unsigned)P.W), px = (int)(r - (unsigned)py * (unsigned)P.W);
    if (P.g_std > 0.0f) adj_ray<DT, TAU, SKIP, true>(P, P.cams, view, px, py, P.iteration + iteration, part, T0);
    else adj_ray<DT, TAU, SKIP, false>(P, P.cams, view, px, py, P.iteration + iteration, part, T0);
}

template <int DT, bool TAU>
__global__ void FR_MARCH_BOUNDS adj_single(const __grid_constant__ SingleArgs a)
{
    adj_body<DT, TAU>(a.p, a.cams, blockIdx.x);
}

// ---------------------------------------------------------------------------
// Exact gradient of the rendered images
// ---------------------------------------------------------------------------

// Along a ray L = sum_k T_k S_k beta_k with T_{k+1} = T_k exp(-sigma_k l_k):
//   dL/dS_k = T_k beta_k,
//   dL/dsigma_k = T_k S_k dbeta_k/dsigma - l_k (L_total - sum_{m<=k} T_m S_m beta_m),
// the suffix sum taken from the rendered L_total.  Per key point the window
// accumulates {dS_r, dS_g, dS_b, dsigma} (RGB) or {dT, dsigma} (temperature).
template <int DT, int KIND, bool TAU>
__device__ __forceinline__ void bwd_body(const ProbDev& P, const CamDev* cams, int tile)
{
    int view, px, py;
    tile_pixel(P, tile, view, px, py);
    if (px >= P.W || py >= P.H) return;
    const long long pix = ((long long)view * P.H + py) * P.W + px;
    const float* gi = P.img_in + 3 * pix;
    const float g0 = gi[0] * P.img_scale, g1 = gi[1] * P.img_scale, g2 = gi[2] * P.img_scale;
    if (g0 == 0.0f && g1 == 0.0f && g2 == 0.0f) return;
    Ray R;
    if (!make_ray(cams[view], px, py, P.nx, P.ny, P.nz, P.step, R)) return;
    const float* lt = P.L_total + 3 * pix;
    const float Lt0 = lt[0], Lt1 = lt[1], Lt2 = lt[2];
    const long long nxy = (long long)P.nx * P.ny;
    using Rec = RecOf<DT, KIND>;
    using RT = typename Rec::T;
    // per key point: {dS_r, dS_g, dS_b, dsigma} (RGB) or {dT, dsigma} (TEMP)
    constexpr int NA = KIND == KIND_RGB ? 4 : 2;
    float acc[8][NA];
    RT v[8];
    long long vbase = -1;
#pragma unroll
    for (int t = 0; t < 8; ++t)
#pragma unroll
        for (int q = 0; q < NA; ++q) acc[t][q] = 0.0f;
    float* dV = P.dV;
    const void* vol = P.vol;
    const long long nodes = nxy * P.nz;
    (void)nodes;
    // (predicated per slot as in the adjustment; reductions of all-zero sums
    // are issued too)
    auto leave = [&acc, dV, nodes](int t, int node, bool p) {
        const unsigned nd = (unsigned)FR_CHK(node, nodes, 2u);
        if constexpr (KIND == KIND_RGB) red_add_v4_if(dV + 4 * nd, acc[t][0], acc[t][1], acc[t][2], acc[t][3], p);
        else red_add_v2_if(dV + 2 * nd, acc[t][0], acc[t][1], p);
#pragma unroll
        for (int q = 0; q < NA; ++q) acc[t][q] = p ? 0.0f : acc[t][q];
    };
    Win W;
    W.live = false;
    float T = 1.0f, p0 = 0.0f, p1 = 0.0f, p2 = 0.0f;
    for (int k = 0; k < R.n; ++k) {
        float len, x, y, z;
        segment(R, P.step, k, len, x, y, z);
        const CellIJK ci = cell_ijk(x, y, z, P.nx, P.ny, P.nz);
        win_move_pred(W, ci.i, ci.j, ci.k, P.nx, P.ny, (int)nxy, leave, [](int, int, bool) {});
        if (W.base != vbase) {
            vbase = W.base;
            load8<DT, KIND>(vol, FR_CHK((long long)W.base, nxy * P.nz - nxy - P.nx - 1, 1u), P.nx, nxy, v);
        }
        const RT r = slot_blend<RT>(v, ci.fx, ci.fy, ci.fz);
        const float gx = mirror_frac(ci.i, ci.fx), gy = mirror_frac(ci.j, ci.fy), gz = mirror_frac(ci.k, ci.fz);
        float S[3], sig, dq[3] = {0.0f, 0.0f, 0.0f};
        if constexpr (KIND == KIND_RGB) record_source<KIND>(P, r, S, sig, dq);
        else record_source_temp(P, r, S, sig, dq);
        float gS0, gS1, gS2, gsig;
        if constexpr (TAU) {
            const float w = T * P.tau;
            gS0 = g0 * w; gS1 = g1 * w; gS2 = g2 * w;
            gsig = 0.0f;
            T *= 1.0f - P.tau;
        } else {
            const float e = __expf(-sig * len);
            const float beta = seg_weight(sig, len, e);
            const float db = seg_weight_dsigma(sig, len, e, beta);
            const float tb = T * beta;
            p0 = fmaf(tb, S[0], p0); p1 = fmaf(tb, S[1], p1); p2 = fmaf(tb, S[2], p2);
            gS0 = g0 * tb; gS1 = g1 * tb; gS2 = g2 * tb;
            const float tdb = T * db;
            gsig = g0 * (tdb * S[0] - len * (Lt0 - p0)) + g1 * (tdb * S[1] - len * (Lt1 - p1)) +
                   g2 * (tdb * S[2] - len * (Lt2 - p2));
            T *= e;
        }
        float gv[NA];
        if constexpr (KIND == KIND_RGB) {
            gv[0] = gS0; gv[1] = gS1; gv[2] = gS2; gv[3] = gsig;
        } else {
            gv[0] = gS0 * dq[0] + gS1 * dq[1] + gS2 * dq[2];
            gv[1] = gsig;
        }
        const float wx[2] = {1.0f - gx, gx}, wy[2] = {1.0f - gy, gy}, wz[2] = {1.0f - gz, gz};
#pragma unroll
        for (int t = 0; t < 8; ++t) {
            const float w = wx[t & 1] * wy[(t >> 1) & 1] * wz[t >> 2];
#pragma unroll
            for (int q = 0; q < NA; ++q) acc[t][q] = fmaf(w, gv[q], acc[t][q]);
        }
    }
    win_release(W, [&leave](int t, int node) { leave(t, node, true); });
}

// Resident CTAs per SM asked for the backward march: 4 with temperature
// records (128 registers), 3 with RGB records (168).
#ifndef FR_BWD_MINB_RGB
#define FR_BWD_MINB_RGB 3
#endif
#ifndef FR_BWD_MINB_TEMP
#define FR_BWD_MINB_TEMP 4
#endif
template <int DT, int KIND, bool TAU>
__global__ void __launch_bounds__(kTileThreads, KIND == KIND_RGB ? FR_BWD_MINB_RGB : FR_BWD_MINB_TEMP)
    bwd_single(const __grid_constant__ SingleArgs a)
{
    const int tile = a.p.tile_order ? (int)__ldg(a.p.tile_order + blockIdx.x) : (int)blockIdx.x;
    bwd_body<DT, KIND, TAU>(a.p, a.cams, tile);
}

template <int DT, int KIND, bool TAU>
__global__ void FR_MARCH_BOUNDS bwd_batch(const ProbDev* __restrict__ probs,
                                                                          const int* __restrict__ tile_start,
                                                                          int nprob)
{
    const int p = find_problem(tile_start, nprob, blockIdx.x);
    const ProbDev& P = probs[p];
    bwd_body<DT, KIND, TAU>(P, P.cams, blockIdx.x - __ldg(tile_start + p));
}

// ---------------------------------------------------------------------------
// Sample counting: segments of every ray (or of the rays with a non-zero
// residual).
// ---------------------------------------------------------------------------

__global__ void __launch_bounds__(kTileThreads) count_single(const __grid_constant__ SingleArgs a)
{
    const ProbDev& P = a.p;
    int view, px, py;
    tile_pixel(P, blockIdx.x, view, px, py);
    unsigned n = 0;
    if (px < P.W && py < P.H) {
        bool use = true;
        if (P.img_in) {
            const float* g = P.img_in + 3 * (((long long)view * P.H + py) * P.W + px);
            use = !(g[0] == 0.0f && g[1] == 0.0f && g[2] == 0.0f);
        }
        Ray R;
        if (use && make_ray(a.cams[view], px, py, P.nx, P.ny, P.nz, P.step, R)) {
            if (P.occ) {
                // the samples the forward march evaluates when it skips empty bricks
                BrickSkip skip;
                for (int k = 0; k < R.n; ++k) {
                    float len, x, y, z;
                    segment(R, P.step, k, len, x, y, z);
                    if (!skip.empty(P.occ, P, R, P.step, x, y, z, k)) ++n;
                }
            } else {
                n = (unsigned)R.n;
            }
        }
    }
    const unsigned s = __reduce_add_sync(0xffffffffu, n);
    if ((threadIdx.x & 31) == 0 && s) atomicAdd(P.counter, (unsigned long long)s);
}

// Deterministic sum of the per-CTA squared-error partials of one problem.
// accumulate != 0: adds to out4 (several views of one pooled error measure).
__global__ void __launch_bounds__(1024) finalize_partials(const float* __restrict__ partials, int ntiles,
                                                          float* __restrict__ out4, int accumulate)
{
    __shared__ float red[4][32];
    float s0 = 0.0f, s1 = 0.0f, s2 = 0.0f, s3 = 0.0f;
    const float4* p4 = reinterpret_cast<const float4*>(partials);
#pragma unroll 4
    for (int i = threadIdx.x; i < ntiles; i += blockDim.x) {
        const float4 v = __ldg(p4 + i);
        s0 += v.x; s1 += v.y; s2 += v.z; s3 += v.w;
    }
    s0 = warp_sum(s0); s1 = warp_sum(s1); s2 = warp_sum(s2); s3 = warp_sum(s3);
    const int w = threadIdx.x >> 5;
    if ((threadIdx.x & 31) == 0) { red[0][w] = s0; red[1][w] = s1; red[2][w] = s2; red[3][w] = s3; }
    __syncthreads();
    if (threadIdx.x < 4) {
        float t = 0.0f;
        for (int i = 0; i < (int)(blockDim.x >> 5); ++i) t += red[threadIdx.x][i];
        out4[threadIdx.x] = accumulate ? out4[threadIdx.x] + t : t;
    }
}

// The same sum over kFinParts CTAs (finalize_parts_body); *done must be 0
// before the first launch.

__global__ void __launch_bounds__(256) finalize_parts(const float* __restrict__ partials, int ntiles,
                                                      float* __restrict__ out4, int accumulate,
                                                      float4* part_sums, unsigned* done, float* rmse3)
{
    finalize_parts_body(partials, ntiles, out4, accumulate, part_sums, done, rmse3, blockIdx.x, gridDim.x);
}

// Flame-ray list (pixels whose prepared target is non-zero), in tile order,
// each tile's run padded to whole warps with entries that name no pixel.
// Pass 1 counts each warp's flame pixels and each CTA's padded total; pass 2
// scans the CTA totals; pass 3 writes each warp's pixels at the CTA offset
// plus the counts of the CTA's earlier warps, and the padding.  Buffer layout:
// warp counts [0, 4 ntiles), CTA offsets [4 ntiles, 5 ntiles], total at
// 5 ntiles (the list holds at most 128 entries per tile).
__device__ __forceinline__ bool is_flame(const ProbDev& P, int view, int px, int py)
{
    if (px >= P.W || py >= P.H) return false;
    const float* t = P.targets + 3 * (((long long)view * P.H + py) * P.W + px);
    return fmaxf(t[0], fmaxf(t[1], t[2])) > P.thresh;
}

constexpr int kWarpsPerTile = kTileThreads / 32;

__global__ void __launch_bounds__(kTileThreads) flame_count_kernel(const __grid_constant__ SingleArgs a,
                                                                   unsigned* __restrict__ buf, int ntiles,
                                                                   unsigned parts)
{
    __shared__ unsigned wc[kWarpsPerTile];
    int view, px, py;
    tile_pixel(a.p, blockIdx.x, view, px, py);
    const unsigned m = __ballot_sync(0xffffffffu, is_flame(a.p, view, px, py));
    const int w = threadIdx.x >> 5;
    if ((threadIdx.x & 31) == 0) {
        wc[w] = __popc(m);
        buf[blockIdx.x * kWarpsPerTile + w] = __popc(m);
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        unsigned t = 0;
        for (int i = 0; i < kWarpsPerTile; ++i) t += wc[i];
        // the run padded to whole warps, once per part of the rays
        buf[(size_t)kWarpsPerTile * ntiles + blockIdx.x] = parts * ((t + 31u) & ~31u);
    }
}

// Exclusive scan of n values in place, total at offsets[n]; one CTA.
__global__ void __launch_bounds__(1024) flame_scan_kernel(unsigned* __restrict__ offsets, int n)
{
    __shared__ unsigned wsum[32];
    __shared__ unsigned carry;
    if (threadIdx.x == 0) carry = 0;
    __syncthreads();
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    for (int base = 0; base < n; base += blockDim.x) {
        const int i = base + threadIdx.x;
        const unsigned v = i < n ? offsets[i] : 0u;
        unsigned x = v;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const unsigned y = __shfl_up_sync(0xffffffffu, x, o);
            if (lane >= o) x += y;
        }
        if (lane == 31) wsum[w] = x;
        __syncthreads();
        if (w == 0) {
            unsigned s = lane < (int)(blockDim.x >> 5) ? wsum[lane] : 0u;
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const unsigned y = __shfl_up_sync(0xffffffffu, s, o);
                if (lane >= o) s += y;
            }
            wsum[lane] = s;  // inclusive
        }
        __syncthreads();
        const unsigned before = carry + (w > 0 ? wsum[w - 1] : 0u) + x - v;
        if (i < n) offsets[i] = before;
        __syncthreads();
        if (threadIdx.x == blockDim.x - 1) carry = before + v;
        __syncthreads();
    }
    if (threadIdx.x == 0) offsets[n] = carry;
}

__global__ void __launch_bounds__(kTileThreads) flame_list_kernel(const __grid_constant__ SingleArgs a,
                                                                  const unsigned* __restrict__ buf, int ntiles,
                                                                  unsigned* __restrict__ list, unsigned parts)
{
    const ProbDev& P = a.p;
    int view, px, py;
    tile_pixel(P, blockIdx.x, view, px, py);
    const bool f = is_flame(P, view, px, py);
    const unsigned m = __ballot_sync(0xffffffffu, f);
    const unsigned run_at = buf[(size_t)kWarpsPerTile * ntiles + blockIdx.x];
    unsigned len = 0;
    for (int i = 0; i < kWarpsPerTile; ++i) len += buf[blockIdx.x * kWarpsPerTile + i];
    const unsigned padded = (len + 31u) & ~31u;
    if (f) {
        const int w = threadIdx.x >> 5;
        unsigned at = run_at;
        for (int i = 0; i < w; ++i) at += buf[blockIdx.x * kWarpsPerTile + i];
        at += __popc(m & ((1u << (threadIdx.x & 31)) - 1u));
        const unsigned pix = (unsigned)(((long long)view * P.H + py) * P.W + px);
        // part j's block of the run: the pixel tagged j in the top two bits
        for (unsigned j = 0; j < parts; ++j) list[at + j * padded] = pix | (j << 30);
    }
    // the run's padding to whole warps names no pixel
    if ((unsigned)threadIdx.x >= len && (unsigned)threadIdx.x < padded)
        for (unsigned j = 0; j < parts; ++j) list[run_at + j * padded + threadIdx.x] = kNoPixel;
}

// Per-problem sums of the squared-error partials (one CTA per problem), into
// the problem's error slot sq_slot + iteration.
__global__ void __launch_bounds__(1024) finalize_batch(const ProbDev* __restrict__ probs, int iteration)
{
    __shared__ float red[4][32];
    const ProbDev& P = probs[blockIdx.x];
    float s0 = 0.0f, s1 = 0.0f, s2 = 0.0f, s3 = 0.0f;
    const float4* p4 = reinterpret_cast<const float4*>(P.partials);
    for (int i = threadIdx.x; i < P.ntiles; i += blockDim.x) {
        const float4 v = __ldg(p4 + i);
        s0 += v.x; s1 += v.y; s2 += v.z; s3 += v.w;
    }
    s0 = warp_sum(s0); s1 = warp_sum(s1); s2 = warp_sum(s2); s3 = warp_sum(s3);
    const int w = threadIdx.x >> 5;
    if ((threadIdx.x & 31) == 0) { red[0][w] = s0; red[1][w] = s1; red[2][w] = s2; red[3][w] = s3; }
    __syncthreads();
    if (threadIdx.x < 4) {
        float t = 0.0f;
        for (int i = 0; i < (int)(blockDim.x >> 5); ++i) t += red[threadIdx.x][i];
        P.sqerr[4 * (P.sq_slot + iteration) + threadIdx.x] = t;
    }
}

// ---------------------------------------------------------------------------
// Host-side dispatch
// ---------------------------------------------------------------------------

#define FR_DISPATCH_DT(dt, DTC, ...)                      \
    switch (dt) {                                         \
        case DT_F32: { constexpr int DTC = DT_F32; __VA_ARGS__; break; }   \
        case DT_BF16: { constexpr int DTC = DT_BF16; __VA_ARGS__; break; } \
        case DT_F16: { constexpr int DTC = DT_F16; __VA_ARGS__; break; }   \
        default: return cudaErrorInvalidValue;            \
    }

cudaError_t launch_tile_order(const SingleArgs& a, int ntiles, const unsigned* box, unsigned* key,
                              unsigned* order, cudaStream_t s)
{
    if (ntiles <= 0) return cudaSuccess;
    tile_work_kernel<<<ntiles, kTileThreads, 0, s>>>(a, box, key);
    tile_order_kernel<<<1, 1024, 0, s>>>(key, ntiles, order);
    return cudaGetLastError();
}

cudaError_t launch_fwd(const SingleArgs& a, int dt, int kind, int ntiles, cudaStream_t s)
{
    const bool tau = a.p.tau > 0.0f;
    const int mode = a.p.pairs == nullptr ? 0 : (a.p.occ != nullptr && kind == KIND_RGB && !tau ? 2 : 1);
    dim3 grid(ntiles), block(kTileThreads);
#define FR_FWD(D, K, T)                                                            \
    if (mode == 2) fwd_single<D, K, T, 2><<<grid, block, 0, s>>>(a);               \
    else if (mode == 1) fwd_single<D, K, T, 1><<<grid, block, 0, s>>>(a);          \
    else fwd_single<D, K, T, 0><<<grid, block, 0, s>>>(a)
    FR_DISPATCH_DT(dt, D, {
        if (kind == KIND_RGB) {
            if (tau) { FR_FWD(D, KIND_RGB, true); } else { FR_FWD(D, KIND_RGB, false); }
        } else {
            if (tau) { FR_FWD(D, KIND_TEMP, true); } else { FR_FWD(D, KIND_TEMP, false); }
        }
    });
#undef FR_FWD
    return cudaGetLastError();
}

cudaError_t preload_noalloc_kernels()
{
    // cudaFuncGetAttributes loads a kernel's module code (lazy loading
    // otherwise loads it, and allocates for it, at the first launch)
    cudaFuncAttributes attr;
    cudaError_t e = cudaFuncGetAttributes(&attr, finalize_partials);
#define FR_PRELOAD(D, K, T) \
    if (e == cudaSuccess) e = cudaFuncGetAttributes(&attr, fwd_single<D, K, T, 0>)
#define FR_PRELOAD_DT(D)                                                                      \
    FR_PRELOAD(D, KIND_RGB, false); FR_PRELOAD(D, KIND_RGB, true); FR_PRELOAD(D, KIND_TEMP, false); \
    FR_PRELOAD(D, KIND_TEMP, true)
    FR_PRELOAD_DT(DT_F32);
    FR_PRELOAD_DT(DT_BF16);
    FR_PRELOAD_DT(DT_F16);
#undef FR_PRELOAD_DT
#undef FR_PRELOAD
    return e;
}

#if FR_FUSED
cudaError_t launch_fused(const SingleArgs& a, int dt, int ntiles, cudaStream_t s)
{
    // the forward's mode 2: x-pair records, brick skipping, no constant tau
    if (a.p.pairs == nullptr || a.p.occ == nullptr || a.p.tau > 0.0f || a.p.flist || a.p.residual)
        return cudaErrorInvalidValue;
    dim3 grid(ntiles), block(kTileThreads);
    FR_DISPATCH_DT(dt, D, {
        if (a.p.adj_occ) fused_single<D, true><<<grid, block, 0, s>>>(a);
        else fused_single<D, false><<<grid, block, 0, s>>>(a);
    });
    return cudaGetLastError();
}
#endif

cudaError_t launch_fwd_batch(const ProbDev* probs, const int* tile_start, int nprob, int total_tiles,
                             int dt, int kind, bool tau, bool pairs, cudaStream_t s, bool skip)
{
    dim3 grid(total_tiles), block(kTileThreads);
    skip = skip && pairs && kind == KIND_RGB && !tau;
#define FR_FWDB(D, K, T)                                                                        \
    if (skip) fwd_batch<D, K, T, 2><<<grid, block, 0, s>>>(probs, tile_start, nprob);            \
    else if (pairs) fwd_batch<D, K, T, 1><<<grid, block, 0, s>>>(probs, tile_start, nprob);      \
    else fwd_batch<D, K, T, 0><<<grid, block, 0, s>>>(probs, tile_start, nprob)
    FR_DISPATCH_DT(dt, D, {
        if (kind == KIND_RGB) {
            if (tau) { FR_FWDB(D, KIND_RGB, true); } else { FR_FWDB(D, KIND_RGB, false); }
        } else {
            if (tau) { FR_FWDB(D, KIND_TEMP, true); } else { FR_FWDB(D, KIND_TEMP, false); }
        }
    });
#undef FR_FWDB
    return cudaGetLastError();
}

cudaError_t launch_adjust(const SingleArgs& a, int dt, int ntiles, cudaStream_t s)
{
    const bool tau = a.p.tau > 0.0f;
    dim3 grid(ntiles), block(kTileThreads);
    FR_DISPATCH_DT(dt, D, {
        if (tau) adj_single<D, true><<<grid, block, 0, s>>>(a);
        else adj_single<D, false><<<grid, block, 0, s>>>(a);
    });
    return cudaGetLastError();
}

cudaError_t launch_adjust_list_batch(const ProbDev* probs, const int* tile_start, int nprob, int total_tiles,
                                     int dt, bool tau, int iteration, cudaStream_t s, bool skip, int parts)
{
    const unsigned np = parts > 1 ? (unsigned)parts : 1u;
    dim3 grid((unsigned)total_tiles * (kTileThreads / FR_ADJ_THREADS) * np), block(FR_ADJ_THREADS);
    FR_DISPATCH_DT(dt, D, {
        if (tau) adj_list_batch<D, true, false><<<grid, block, 0, s>>>(probs, tile_start, nprob, iteration, np);
        else if (skip) adj_list_batch<D, false, true><<<grid, block, 0, s>>>(probs, tile_start, nprob, iteration, np);
        else adj_list_batch<D, false, false><<<grid, block, 0, s>>>(probs, tile_start, nprob, iteration, np);
    });
    return cudaGetLastError();
}

cudaError_t launch_finalize_batch(const ProbDev* probs, int nprob, int iteration, cudaStream_t s)
{
    finalize_batch<<<nprob, 1024, 0, s>>>(probs, iteration);
    return cudaGetLastError();
}

cudaError_t launch_backward(const SingleArgs& a, int dt, int kind, int ntiles, cudaStream_t s)
{
    const bool tau = a.p.tau > 0.0f;
    dim3 grid(ntiles), block(kTileThreads);
    FR_DISPATCH_DT(dt, D, {
        if (kind == KIND_RGB) {
            if (tau) bwd_single<D, KIND_RGB, true><<<grid, block, 0, s>>>(a);
            else bwd_single<D, KIND_RGB, false><<<grid, block, 0, s>>>(a);
        } else {
            if (tau) bwd_single<D, KIND_TEMP, true><<<grid, block, 0, s>>>(a);
            else bwd_single<D, KIND_TEMP, false><<<grid, block, 0, s>>>(a);
        }
    });
    return cudaGetLastError();
}

cudaError_t launch_backward_batch(const ProbDev* probs, const int* tile_start, int nprob, int total_tiles,
                                  int dt, int kind, bool tau, cudaStream_t s)
{
    dim3 grid(total_tiles), block(kTileThreads);
    FR_DISPATCH_DT(dt, D, {
        if (kind == KIND_RGB) {
            if (tau) bwd_batch<D, KIND_RGB, true><<<grid, block, 0, s>>>(probs, tile_start, nprob);
            else bwd_batch<D, KIND_RGB, false><<<grid, block, 0, s>>>(probs, tile_start, nprob);
        } else {
            if (tau) bwd_batch<D, KIND_TEMP, true><<<grid, block, 0, s>>>(probs, tile_start, nprob);
            else bwd_batch<D, KIND_TEMP, false><<<grid, block, 0, s>>>(probs, tile_start, nprob);
        }
    });
    return cudaGetLastError();
}

cudaError_t launch_count(const SingleArgs& a, int ntiles, cudaStream_t s)
{
    count_single<<<ntiles, kTileThreads, 0, s>>>(a);
    return cudaGetLastError();
}

cudaError_t launch_finalize(const float* partials, int ntiles, float* out4, cudaStream_t s, int accumulate,
                            void* scratch, float* rmse3)
{
    if (scratch) {
        float4* part_sums = reinterpret_cast<float4*>(scratch);
        unsigned* done = reinterpret_cast<unsigned*>(part_sums + kFinParts);
        finalize_parts<<<kFinParts, 256, 0, s>>>(partials, ntiles, out4, accumulate, part_sums, done, rmse3);
    } else {
        finalize_partials<<<1, 1024, 0, s>>>(partials, ntiles, out4, accumulate);
    }
    return cudaGetLastError();
}

cudaError_t launch_flame_list(const SingleArgs& a, int ntiles, unsigned* buf, unsigned* list, cudaStream_t s,
                              int parts)
{
    const unsigned np = parts > 1 ? (unsigned)parts : 1u;
    flame_count_kernel<<<ntiles, kTileThreads, 0, s>>>(a, buf, ntiles, np);
    flame_scan_kernel<<<1, 1024, 0, s>>>(buf + (size_t)kWarpsPerTile * ntiles, ntiles);
    flame_list_kernel<<<ntiles, kTileThreads, 0, s>>>(a, buf, ntiles, list, np);
    return cudaGetLastError();
}

cudaError_t launch_adjust_list(const SingleArgs& a, int dt, int ntiles, const unsigned* list,
                               const unsigned* count, cudaStream_t s, const float* tm)
{
    static_assert(FR_ADJ_THREADS % 32 == 0 && kTileThreads % FR_ADJ_THREADS == 0, "adjustment CTA size");
    const bool tau = a.p.tau > 0.0f;
#if FR_ADJ_SPLIT > 1
    const unsigned parts = tm ? (unsigned)FR_ADJ_SPLIT : 1u;
#else
    const unsigned parts = 1u;
#endif
    dim3 grid((unsigned)ntiles * (kTileThreads / FR_ADJ_THREADS) * parts), block(FR_ADJ_THREADS);
    const bool skip = a.p.adj_occ != nullptr && !tau;
#if FR_ADJ_ACCUM == 1
    FR_DISPATCH_DT(dt, D, {
        if (tau) adj_list_tab<D, true, false><<<grid, block, 0, s>>>(a, list, count, tm);
        else if (skip) adj_list_tab<D, false, true><<<grid, block, 0, s>>>(a, list, count, tm);
        else adj_list_tab<D, false, false><<<grid, block, 0, s>>>(a, list, count, tm);
    });
#else
    FR_DISPATCH_DT(dt, D, {
        if (tau) adj_list<D, true, false><<<grid, block, 0, s>>>(a, list, count, tm);
        else if (skip) adj_list<D, false, true><<<grid, block, 0, s>>>(a, list, count, tm);
        else adj_list<D, false, false><<<grid, block, 0, s>>>(a, list, count, tm);
    });
#endif
    return cudaGetLastError();
}

#ifdef FR_ADJ_GATHER_PROBE
// Measurement of the gather form of the adjustment (one thread per key point
// summing over the rays that sample its eight cells), built only with
// -DFR_ADJ_GATHER_PROBE.  A gather evaluates the same (sample, key point)
// pairs as the scatter, but before any of them it must find, per key point
// and view, the flame pixels whose rays can cross the box of its eight cells
// and each such ray's samples inside that box.  gather_probe_kernel does that
// set-up work alone -- the box's projection, the residual test of every pixel
// in its rectangle, the ray and its clip to the box -- and none of the
// per-sample work (positions, cells, distance weights, the transmittance a
// gather would have to read from a store the forward march wrote): its time is
// a lower bound on any gather's.  Its output (a sample count weighted by the
// red residual per key point) is discarded.
__global__ void __launch_bounds__(256) hull_nodes_kernel(const unsigned* __restrict__ tags, long long nodes,
                                                         unsigned full, unsigned* __restrict__ list,
                                                         unsigned* __restrict__ count)
{
    const long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    const bool in = i < nodes && __ldg(tags + i) == full;
    const unsigned m = __ballot_sync(0xffffffffu, in);
    const int lane = threadIdx.x & 31;
    unsigned base = 0;
    if (lane == 0 && m) base = atomicAdd(count, (unsigned)__popc(m));
    base = __shfl_sync(0xffffffffu, base, 0);
    if (in) list[base + __popc(m & ((1u << lane) - 1u))] = (unsigned)i;
}

__global__ void __launch_bounds__(128) gather_probe_kernel(const __grid_constant__ SingleArgs a,
                                                           const unsigned* __restrict__ list,
                                                           const unsigned* __restrict__ count,
                                                           float* __restrict__ sink)
{
    const unsigned t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= __ldg(count)) return;
    const ProbDev& P = a.p;
    const unsigned node = __ldg(list + t);
    const int nx = P.nx, ny = P.ny, nz = P.nz;
    const int i = (int)(node % (unsigned)nx), j = (int)((node / (unsigned)nx) % (unsigned)ny),
              k = (int)(node / ((unsigned)nx * (unsigned)ny));
    const float lo[3] = {(float)max(i - 1, 0), (float)max(j - 1, 0), (float)max(k - 1, 0)};
    const float hi[3] = {(float)min(i + 1, nx - 1), (float)min(j + 1, ny - 1), (float)min(k + 1, nz - 1)};
    float sum = 0.0f;
    for (int v = 0; v < P.ncam; ++v) {
        const CamDev& c = a.cams[v];
        float umin = INFINITY, umax = -INFINITY, wmin = INFINITY, wmax = -INFINITY;
        bool behind = false;
#pragma unroll
        for (int b = 0; b < 8; ++b) {
            const float X = ((b & 1) ? hi[0] : lo[0]) - c.o[0], Y = ((b & 2) ? hi[1] : lo[1]) - c.o[1],
                        Z = ((b & 4) ? hi[2] : lo[2]) - c.o[2];
            const float xc = X * c.r[0] + Y * c.r[1] + Z * c.r[2], yc = X * c.u[0] + Y * c.u[1] + Z * c.u[2];
            const float zc = X * c.f[0] + Y * c.f[1] + Z * c.f[2];
            behind |= !(zc > 0.0f);
            const float u = (xc / zc / c.tx + 1.0f) * 0.5f * (float)c.W - 0.5f;
            const float w = (1.0f - yc / zc / c.ty) * 0.5f * (float)c.H - 0.5f;
            umin = fminf(umin, u); umax = fmaxf(umax, u); wmin = fminf(wmin, w); wmax = fmaxf(wmax, w);
        }
        if (behind) continue;
        const int x0 = max((int)ceilf(umin), 0), x1 = min((int)floorf(umax), c.W - 1);
        const int y0 = max((int)ceilf(wmin), 0), y1 = min((int)floorf(wmax), c.H - 1);
        for (int py = y0; py <= y1; ++py)
            for (int px = x0; px <= x1; ++px) {
                const long long pix = ((long long)v * c.H + py) * c.W + px;
                const float r0 = __ldg(P.img_in + 3 * pix), r1 = __ldg(P.img_in + 3 * pix + 1),
                            r2 = __ldg(P.img_in + 3 * pix + 2);
                if (r0 == 0.0f && r1 == 0.0f && r2 == 0.0f) continue;
                Ray R;
                if (!make_ray(c, px, py, nx, ny, nz, P.step, R)) continue;
                const float o[3] = {R.p0x, R.p0y, R.p0z}, id[3] = {R.idx, R.idy, R.idz}, d[3] = {R.dx, R.dy, R.dz};
                float tin = 0.0f, tout = R.chord;
#pragma unroll
                for (int ax = 0; ax < 3; ++ax) {
                    if (d[ax] == 0.0f) continue;
                    const float t0 = (lo[ax] - o[ax]) * id[ax], t1 = (hi[ax] - o[ax]) * id[ax];
                    tin = fmaxf(tin, fminf(t0, t1));
                    tout = fminf(tout, fmaxf(t0, t1));
                }
                if (tout < tin) continue;
                const int ka = max(0, (int)ceilf(tin / P.step - 0.5f) - 1);
                const int kb = min(R.n - 1, (int)floorf(tout / P.step) + 1);
                sum += (float)(kb - ka + 1) * r0;
            }
    }
    sink[node] = sum;
}

cudaError_t launch_gather_probe(const SingleArgs& a, const unsigned* tags, unsigned full, long long nodes,
                                unsigned* list, unsigned* count, float* sink, cudaStream_t s)
{
    cudaError_t e = cudaMemsetAsync(count, 0, sizeof(unsigned), s);
    if (e != cudaSuccess) return e;
    hull_nodes_kernel<<<(unsigned)((nodes + 255) / 256), 256, 0, s>>>(tags, nodes, full, list, count);
    gather_probe_kernel<<<(unsigned)((nodes + 127) / 128), 128, 0, s>>>(a, list, count, sink);
    return cudaGetLastError();
}
#endif

// The check word of this translation unit (0 in the normal build).
cudaError_t check_word_march(unsigned* word, bool reset)
{
#ifdef FR_CHECKED
    cudaError_t e = cudaMemcpyFromSymbol(word, g_fr_check_word, sizeof(unsigned));
    if (e == cudaSuccess && reset) {
        const unsigned zero = 0;
        e = cudaMemcpyToSymbol(g_fr_check_word, &zero, sizeof(unsigned));
    }
    return e;
#else
    (void)reset;
    *word = 0;
    return cudaSuccess;
#endif
}

}  // namespace frk
