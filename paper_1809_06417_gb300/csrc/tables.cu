// tables.cu -- the paper-rule loop over a fixed extinction field as two
// sparse linear maps, built once per reconstruction call.
//
// The paper rule (Eqs. 10-11) adjusts the key points' colours only and keeps
// sigma_t fixed (Sec. 3.3.1 takes it constant); with G(s) = 1 (Eq. 11) the
// transmittance at every sample of every ray is then the same at every
// iteration, and both halves of an iteration of Algorithm 2 are linear maps
// whose coefficients do not change:
//   * rendering (Eqs. 5-8): the radiance of pixel p is
//       L_p = sum_j A_pj S_j,   A_pj = sum_s T(s) beta(s) w_j(s),
//     over the samples s of p's ray, T(s) the transmittance in front of s,
//     beta(s) = (1 - e^{-sigma l}) / sigma its segment weight and w_j(s) the
//     trilinear weight of key point j at s (S_j: source record of j);
//   * adjustment (Eq. 10): key point j moves by
//       dV_j = sum_p W_pj dL_p,  W_pj = sum_s alpha_l T(s) e^{-alpha_d D(j, s)},
//     over the flame rays p and their samples s whose cell has j as a corner.
// One march over every ray fills both tables with an entry for each (ray, key
// point inside the visual hull) pair -- records outside the hull are zero and
// their updates are discarded (Sec. 4.3.1) -- and every iteration then streams
// them: the forward table ray by ray (a gather of source records), the
// adjustment table key point by key point (a gather of the flame rays'
// residuals: the per-key-point gather form of the adjustment, no atomics).
//
// Layouts.  The hull's key points are listed in Morton (Z) order of their
// node coordinates (node order when the grid is far from cubic): hnode[h] is
// the node of list entry h, and each iteration copies the source records of
// the list into hs[h] first, so that the key points a bundle of neighbouring
// rays samples lie close together in memory.  Forward table: warp w (one of
// the four 8 x 4 sub-tiles of a 16 x 8 pixel tile, as in the marches) owns
// rows [woff[w], woff[w] + wrows[w]); row r holds one entry per lane at
// 32 r + lane, {h, A as float bits}; a lane's rows after its last entry hold
// {0, 0}.  Flame rays are numbered in tile order (the tile's offset tfoff
// plus the ray's rank among the tile's flame pixels).  Adjustment table: key
// point h of the hull list owns entries [hend[h - 1], hend[h]) of
// {flame-ray number, W as float bits}, in the order the fill pass's atomics
// hand out (built with FR_TAB_SORT = 1: in increasing flame-ray order).
#include <algorithm>
#include <vector>

#include "fr_device.cuh"
#include "fr_internal.h"

namespace frk {

namespace {

// One ray's march over the samples in bricks holding a key point inside the
// hull (the adjustment's skipping, exact for both tables), with the
// parity-slot window of the adjustment: emit(node, A, W) runs for each key
// point of the hull the ray leaves, with its two sums (sums = false: the
// same key points, the sums left at 0).  W is accumulated for flame rays
// only.  The sample positions, cells and transmittance are those
// of the paper-rule adjustment march (adj_ray), so the same key points
// receive the same samples.
template <int DT, class Emit>
__device__ __forceinline__ void tab_march(const ProbDev& P, const CamDev& cam, int px, int py, bool flame,
                                          const unsigned* __restrict__ tags, unsigned full, bool sums,
                                          Emit&& emit)
{
    Ray R;
    if (!make_ray(cam, px, py, P.nx, P.ny, P.nz, P.step, R)) return;
    int k0 = 0, k1 = R.n;
    if (!BrickSkip::box_range(P, P.adj_box, R, P.step, k0, k1)) return;
    const long long nodes = (long long)P.nx * P.ny * P.nz;
    (void)nodes;
    const int nxy32 = P.nx * P.ny;
    const float dcoef = -P.alpha_d * kLog2e;
    float A[8], Wt[8], sg[8];
#pragma unroll
    for (int t = 0; t < 8; ++t) { A[t] = 0.0f; Wt[t] = 0.0f; sg[t] = 0.0f; }
    auto leave = [&](int t, int node, bool p) {
        if (p) {
            if (__ldg(tags + FR_CHK(node, nodes, 32u)) == full) emit(node, A[t], Wt[t]);
            A[t] = 0.0f;
            Wt[t] = 0.0f;
        }
    };
    auto enter = [&](int t, int node, bool p) {
        if (p && sums) sg[t] = load_rgb_sigma<DT>(P.vol, FR_CHK(node, nodes, 1u));
    };
    Win W;
    W.live = false;
    BrickSkip skip;
    float T = 1.0f;
    for (int k = k0; k < k1; ++k) {
        float len, x, y, z;
        segment(R, P.step, k, len, x, y, z);
        const CellIJK c = cell_ijk(x, y, z, P.nx, P.ny, P.nz);
        if (skip.empty_at(P.adj_occ, P, R, P.step, c, k)) continue;
        win_move_pred(W, c.i, c.j, c.k, P.nx, P.ny, nxy32, leave, enter);
        if (!sums) continue;   // (the count pass: which key points, not their sums)
        const float gx = mirror_frac(c.i, c.fx), gy = mirror_frac(c.j, c.fy), gz = mirror_frac(c.k, c.fz);
        const float sig = slot_blend<float>(sg, gx, gy, gz);
        const float e = __expf(-sig * len);
        const float beta = T * seg_weight(sig, len, e);
        // trilinear weight of slot t: (t & 1 ? gx : 1 - gx) (t & 2 ? gy : 1 - gy) (t & 4 ? gz : 1 - gz)
        const float wx[2] = {1.0f - gx, gx}, wy[2] = {1.0f - gy, gy}, wz[2] = {1.0f - gz, gz};
#pragma unroll
        for (int t = 0; t < 8; ++t) A[t] = fmaf(beta, wx[t & 1] * wy[(t >> 1) & 1] * wz[t >> 2], A[t]);
        if (flame) {
            const float base = P.alpha_l * T;
            // squared distances (voxel units) from the sample to each slot's key point
            const float ex[2] = {gx * gx, (1.0f - gx) * (1.0f - gx)};
            const float ey[2] = {gy * gy, (1.0f - gy) * (1.0f - gy)};
            const float ez[2] = {gz * gz, (1.0f - gz) * (1.0f - gz)};
#pragma unroll
            for (int t = 0; t < 8; ++t)
                Wt[t] = fmaf(base, dist_weight(dcoef, ex[t & 1] + ey[(t >> 1) & 1] + ez[t >> 2]), Wt[t]);
        }
        T *= e;
    }
    win_release(W, [&](int t, int node) { leave(t, node, true); });
}

__device__ __forceinline__ bool flame_pixel(const ProbDev& P, long long pix)
{
    const float* t = P.targets + 3 * pix;
    return fmaxf(__ldg(t), fmaxf(__ldg(t + 1), __ldg(t + 2))) > P.thresh;
}

// One kernel for both passes, so that the two run the same instructions and
// emit the same entries.  Count pass (fill = 0): entries per ray (their
// warp's maximum: the warp's rows), flame rays per tile, and the adjustment
// entries of every key point (ncnt, zeroed beforehand).  Fill pass (fill =
// 1): the entries themselves, ncnt holding each key point's next free
// adjustment entry; writes past the counted rows or entries are dropped.
#ifndef FR_TAB_BUILD_MINB
#define FR_TAB_BUILD_MINB 0
#endif
#if FR_TAB_BUILD_MINB
#define FR_TAB_BUILD_BOUNDS __launch_bounds__(kTileThreads, FR_TAB_BUILD_MINB)
#else
#define FR_TAB_BUILD_BOUNDS __launch_bounds__(kTileThreads)
#endif
template <int DT>
__global__ void FR_TAB_BUILD_BOUNDS tab_build_kernel(const __grid_constant__ SingleArgs a, TabBuild b, int fill)
{
    const ProbDev& P = a.p;
    // the tiles longest first (b.torder: estimated for the count, from the
    // count's rows for the fill)
    const unsigned tile = b.torder ? __ldg(b.torder + blockIdx.x) : blockIdx.x;
    int view, px, py;
    tile_pixel(P, (int)tile, view, px, py);
    const bool valid = px < P.W && py < P.H;
    const long long pix = ((long long)view * P.H + py) * P.W + px;
    const bool flame = valid && flame_pixel(P, pix);
    __shared__ unsigned wc[kTileThreads / 32];
    const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const unsigned wi = tile * (kTileThreads / 32) + w;
    unsigned fid = 0, rows = 0;
    uint2* out = nullptr;
    if (fill) {
        // the flame ray's number: the tile's offset and its rank in the tile
        const unsigned m = __ballot_sync(0xffffffffu, flame);
        if (lane == 0) wc[w] = (unsigned)__popc(m);
        __syncthreads();
        fid = __ldg(b.tfoff + tile) + (unsigned)__popc(m & ((1u << lane) - 1u));
        for (int i = 0; i < w; ++i) fid += wc[i];
        rows = __ldg(b.wrows + wi);
        out = b.efwd + (size_t)__ldg(b.woff + wi) * 32 + lane;
    }
    unsigned n = 0;
    if (valid)
        tab_march<DT>(P, a.cams[view], px, py, flame, b.tags, b.full, fill != 0, [&](int node, float A, float W) {
            if (fill) {
                if (n < rows) out[(size_t)n * 32] = make_uint2(__ldg(b.hid + node), __float_as_uint(A));
                if (flame) {
                    const unsigned at = atomicAdd(b.ncnt + node, 1u);
                    if (at < b.nadj) b.eadj[at] = make_uint2(fid, __float_as_uint(W));
                }
            } else if (flame) {
                atomicAdd(b.ncnt + node, 1u);
            }
            ++n;
        });
    if (fill) {
        // padding: the hull's first key point with weight 0
        for (; n < rows; ++n) out[(size_t)n * 32] = make_uint2(0u, 0u);
    } else {
        n = __reduce_max_sync(0xffffffffu, n);
        const int nflame = __syncthreads_count(flame);
        if (lane == 0) b.wrows[wi] = n;
        if (threadIdx.x == 0) b.tfl[tile] = (unsigned)nflame;
    }
}

// ---------------------------------------------------------------------------
// Exclusive scans (block sums, a one-CTA scan of them, then each block's
// items), 64-bit running sums
// ---------------------------------------------------------------------------

constexpr int kScanThreads = 1024;
constexpr int kScanItems = 4;
constexpr int kScanChunk = kScanThreads * kScanItems;

__device__ __forceinline__ unsigned long long block_excl_scan(unsigned long long v, unsigned long long* total)
{
    __shared__ unsigned long long ws[kScanThreads / 32];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    unsigned long long x = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const unsigned long long y = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= o) x += y;
    }
    if (lane == 31) ws[w] = x;
    __syncthreads();
    if (w == 0) {
        unsigned long long s = ws[lane];
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const unsigned long long y = __shfl_up_sync(0xffffffffu, s, o);
            if (lane >= o) s += y;
        }
        ws[lane] = s;
    }
    __syncthreads();
    const unsigned long long before = (w ? ws[w - 1] : 0ull) + x - v;
    if (total) *total = ws[kScanThreads / 32 - 1];
    __syncthreads();
    return before;
}

// Scan inputs: the value of item i.
struct GetU32 {
    const unsigned* v;
    __device__ unsigned operator()(long long i) const { return __ldg(v + i); }
};
// per key point in the listing order: its adjustment entries, whether it is inside the hull
struct GetCountOrdered {
    const unsigned* ncnt;
    KeyOrder o;
    __device__ unsigned operator()(long long i) const
    {
        const long long n = o.node(i);
        return n < 0 ? 0u : __ldg(ncnt + n);
    }
};
struct GetInHullOrdered {
    const unsigned* tags;
    unsigned full;
    KeyOrder o;
    __device__ unsigned operator()(long long i) const
    {
        const long long n = o.node(i);
        return n >= 0 && __ldg(tags + n) == full ? 1u : 0u;
    }
};
// Scan outputs: item i with its exclusive prefix `at` and value v.
struct PutU32 {
    unsigned* out;
    __device__ void operator()(long long i, unsigned long long at, unsigned) const { out[i] = (unsigned)at; }
};
struct PutCursorOrdered {
    unsigned* ncnt;
    KeyOrder o;
    __device__ void operator()(long long i, unsigned long long at, unsigned) const
    {
        const long long n = o.node(i);
        if (n >= 0) ncnt[n] = (unsigned)at;
    }
};
struct PutCompactOrdered {
    unsigned* list;
    KeyOrder o;
    __device__ void operator()(long long i, unsigned long long at, unsigned v) const
    {
        if (v) list[at] = (unsigned)o.node(i);
    }
};

template <class Get>
__global__ void __launch_bounds__(kScanThreads) scan_sums_kernel(Get get, long long n, unsigned long long* bsum)
{
    const long long i0 = (long long)blockIdx.x * kScanChunk + (long long)threadIdx.x * kScanItems;
    unsigned long long s = 0;
#pragma unroll
    for (int q = 0; q < kScanItems; ++q)
        if (i0 + q < n) s += get(i0 + q);
    unsigned long long total;
    block_excl_scan(s, &total);
    if (threadIdx.x == 0) bsum[blockIdx.x] = total;
}

// one CTA: bsum[0 .. nb) to exclusive prefixes, the sum to *total
__global__ void __launch_bounds__(kScanThreads) scan_top_kernel(unsigned long long* bsum, int nb,
                                                                unsigned long long* total)
{
    unsigned long long carry = 0;
    for (int base = 0; base < nb; base += kScanThreads) {
        const int i = base + threadIdx.x;
        const unsigned long long v = i < nb ? bsum[i] : 0ull;
        unsigned long long t;
        const unsigned long long before = block_excl_scan(v, &t);
        if (i < nb) bsum[i] = carry + before;
        carry += t;
    }
    if (threadIdx.x == 0) *total = carry;
}

template <class Get, class Put>
__global__ void __launch_bounds__(kScanThreads) scan_put_kernel(Get get, Put put, long long n,
                                                                const unsigned long long* bsum)
{
    const long long i0 = (long long)blockIdx.x * kScanChunk + (long long)threadIdx.x * kScanItems;
    unsigned v[kScanItems];
    unsigned long long s = 0;
#pragma unroll
    for (int q = 0; q < kScanItems; ++q) {
        v[q] = i0 + q < n ? get(i0 + q) : 0u;
        s += v[q];
    }
    unsigned long long at = bsum[blockIdx.x] + block_excl_scan(s, nullptr);
#pragma unroll
    for (int q = 0; q < kScanItems; ++q) {
        if (i0 + q < n) put(i0 + q, at, v[q]);
        at += v[q];
    }
}

template <class Get, class Put>
cudaError_t scan(Get get, Put put, long long n, unsigned long long* bsum, unsigned long long* total, cudaStream_t s)
{
    const int nb = (int)((n + kScanChunk - 1) / kScanChunk);
    if (nb == 0) return cudaMemsetAsync(total, 0, sizeof *total, s);
    scan_sums_kernel<<<nb, kScanThreads, 0, s>>>(get, n, bsum);
    scan_top_kernel<<<1, kScanThreads, 0, s>>>(bsum, nb, total);
    scan_put_kernel<<<nb, kScanThreads, 0, s>>>(get, put, n, bsum);
    return cudaGetLastError();
}

// hid[hnode[h]] = h for the *count key points of the hull
__global__ void __launch_bounds__(256) hid_kernel(const unsigned* __restrict__ hnode,
                                                  const unsigned long long* __restrict__ count, unsigned* __restrict__ hid)
{
    const unsigned long long h = blockIdx.x * 256ull + threadIdx.x;
    if (h < *count) hid[__ldg(hnode + h)] = (unsigned)h;
}

// The records the forward gathers, for the hull's key points in the list's
// order: hs[h] = records[hnode[h]] (R: the record's bytes as one vector).
template <class R>
__global__ void __launch_bounds__(256) stage_kernel(const R* __restrict__ rec, const unsigned* __restrict__ hnode,
                                                    unsigned nh, R* __restrict__ hs)
{
    const unsigned h = blockIdx.x * 256u + threadIdx.x;
    if (h < nh) hs[h] = __ldg(rec + __ldg(hnode + h));
}

__global__ void __launch_bounds__(256) hend_kernel(const unsigned* __restrict__ hnode, const unsigned* __restrict__ cursor,
                                                   unsigned nh, unsigned* __restrict__ hend)
{
    const unsigned h = blockIdx.x * 256u + threadIdx.x;
    if (h < nh) hend[h] = __ldg(cursor + __ldg(hnode + h));
}

// Each key point's adjustment entries in increasing flame-ray order (the fill
// pass appends them in the order its atomics return): one warp per key point
// sorts its entries in shared memory by a bitonic network over the next power
// of two (padding keys sort last).  A flame ray names a key point once (the
// eight cells around it form a convex box, which a ray enters and leaves
// once), so the order is unique.  Key points with more than kSortMax entries
// keep their order.
constexpr int kSortMax = 512;
constexpr int kSortWarps = 8;
__global__ void __launch_bounds__(32 * kSortWarps) tab_sort_kernel(uint2* __restrict__ eadj,
                                                                  const unsigned* __restrict__ hend, unsigned nh)
{
    __shared__ uint2 buf[kSortWarps][kSortMax];
    const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const unsigned g = blockIdx.x * (unsigned)kSortWarps + w;
    if (g >= nh) return;
    const unsigned b = g ? __ldg(hend + g - 1) : 0u, e = __ldg(hend + g), n = e - b;
    if (n <= 1 || n > (unsigned)kSortMax) return;
    unsigned P = 32;
    while (P < n) P <<= 1;
    uint2* B = buf[w];
    for (unsigned i = lane; i < P; i += 32) B[i] = i < n ? eadj[b + i] : make_uint2(0xffffffffu, 0u);
    __syncwarp();
    for (unsigned k = 2; k <= P; k <<= 1) {
        for (unsigned j = k >> 1; j > 0; j >>= 1) {
            for (unsigned i = lane; i < P; i += 32) {
                const unsigned l = i ^ j;
                if (l > i) {
                    const uint2 x = B[i], y = B[l];
                    const bool up = (i & k) == 0;
                    if ((x.x > y.x) == up) {
                        B[i] = y;
                        B[l] = x;
                    }
                }
            }
            __syncwarp();
        }
    }
    for (unsigned i = lane; i < n; i += 32) eadj[b + i] = B[i];
}

// ---------------------------------------------------------------------------
// Per iteration
// ---------------------------------------------------------------------------

#ifndef FR_TAB_UNROLL
#define FR_TAB_UNROLL 4
#endif
constexpr int kTabUnroll = FR_TAB_UNROLL;
#ifndef FR_TAB_ADJ_UNROLL
#define FR_TAB_ADJ_UNROLL FR_TAB_UNROLL
#endif
constexpr int kTabAdjUnroll = FR_TAB_ADJ_UNROLL;
// CTAs per SM the forward is compiled for (0: no bound)
#ifndef FR_TAB_FWD_MINB
#define FR_TAB_FWD_MINB 0
#endif
#if FR_TAB_FWD_MINB
#define FR_TAB_FWD_BOUNDS __launch_bounds__(kTileThreads, FR_TAB_FWD_MINB)
#else
#define FR_TAB_FWD_BOUNDS __launch_bounds__(kTileThreads)
#endif
// rows ahead of the current group whose entries are prefetched into L2 (0: none)
#ifndef FR_TAB_PREFETCH
#define FR_TAB_PREFETCH 16
#endif
// rows per bulk L2 prefetch of a warp's forward entries (one
// cp.async.bulk.prefetch per chunk, a chunk ahead; 0: none)
#ifndef FR_TAB_BULK
#define FR_TAB_BULK 0
#endif
// 1: each warp of the adjustment prefetches its key points' entries into L2
// with one bulk prefetch before it starts
#ifndef FR_TAB_ADJ_BULK
#define FR_TAB_ADJ_BULK 0
#endif

// L2 prefetch of `bytes` (a multiple of 16) from a 16-byte aligned address by
// the bulk-copy unit (no completion to wait for)
__device__ __forceinline__ void bulk_prefetch_l2(const void* p, unsigned bytes)
{
    asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;" ::"l"(p), "r"(bytes) : "memory");
}

// Forward: each lane sums its ray's entries, A times the entry's source record
// (rows read once per iteration: streaming loads that leave the L2 to the
// records), then the forward march's epilogue: rendered image and residual
// image when asked for, each flame ray's residual at its number, the tile's
// squared-error partials.
template <int DT>
__device__ __forceinline__ void tab_forward_body(const ProbDev& P, const TabIter& it, unsigned slot)
{
    int view, px, py;
    // the tiles in the order of it.torder (longest first, so the grid ends on short ones)
    const unsigned tile = it.torder ? __ldg(it.torder + slot) : slot;
    tile_pixel(P, (int)tile, view, px, py);
    const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const unsigned wi = tile * (kTileThreads / 32) + w;
    const unsigned rows = __ldg(it.wrows + wi);
    const uint2* E = it.efwd + (size_t)__ldg(it.woff + wi) * 32 + lane;
    const long long nodes = (long long)P.nx * P.ny * P.nz;
    (void)nodes;
    // rows streamed kTabUnroll at a time, the next group's entries loaded
    // before this group's records are gathered (two dependent loads in
    // flight per row instead of one after the other)
    float L0 = 0.0f, L1 = 0.0f, L2 = 0.0f;
#if FR_TAB_BULK
    static_assert(FR_TAB_BULK % FR_TAB_UNROLL == 0, "bulk prefetch chunks hold whole groups");
    const char* Erow = reinterpret_cast<const char*>(it.efwd + (size_t)__ldg(it.woff + wi) * 32);
    if (lane == 0 && rows) bulk_prefetch_l2(Erow, min(rows, 2u * FR_TAB_BULK) * 256u);
#endif
    uint2 cur[kTabUnroll];
#pragma unroll
    for (int q = 0; q < kTabUnroll; ++q) cur[q] = (unsigned)q < rows ? __ldcs(E + (size_t)q * 32) : make_uint2(0u, 0u);
    for (unsigned r = 0; r < rows; r += kTabUnroll) {
#if FR_TAB_BULK
        // at each chunk start, the chunk after the next one
        if (lane == 0 && r % FR_TAB_BULK == 0 && r + 2u * FR_TAB_BULK < rows)
            bulk_prefetch_l2(Erow + (size_t)(r + 2u * FR_TAB_BULK) * 256u,
                             min(rows - (r + 2u * FR_TAB_BULK), (unsigned)FR_TAB_BULK) * 256u);
#endif
        uint2 nxt[kTabUnroll];
#pragma unroll
        for (int q = 0; q < kTabUnroll; ++q) {
            const unsigned rr = r + kTabUnroll + q;
            nxt[q] = rr < rows ? __ldcs(E + (size_t)rr * 32) : make_uint2(0u, 0u);
        }
#if FR_TAB_PREFETCH
#pragma unroll
        for (int q = 0; q < kTabUnroll; ++q) {
            const unsigned rr = r + FR_TAB_PREFETCH + q;
            if (rr < rows) asm volatile("prefetch.global.L2 [%0];" ::"l"(E + (size_t)rr * 32));
        }
#endif
        float4 v[kTabUnroll];
#pragma unroll
        for (int q = 0; q < kTabUnroll; ++q)
            v[q] = r + q < rows ? load_rgb<DT>(it.hs, FR_CHK(cur[q].x, it.nhull, 1u)) : make_float4(0.0f, 0.0f, 0.0f, 0.0f);
#pragma unroll
        for (int q = 0; q < kTabUnroll; ++q) {
            const float A = __uint_as_float(cur[q].y);
            L0 = fmaf(A, v[q].x, L0); L1 = fmaf(A, v[q].y, L1); L2 = fmaf(A, v[q].z, L2);
            cur[q] = nxt[q];
        }
    }
    const bool valid = px < P.W && py < P.H;
    const long long pix = valid ? FR_CHK(((long long)view * P.H + py) * P.W + px, (long long)P.ncam * P.H * P.W, 4u)
                                : 0;
    float a0 = 0.0f, a1 = 0.0f, a2 = 0.0f, cnt = 0.0f;
    float d0 = 0.0f, d1 = 0.0f, d2 = 0.0f;
    bool flame = false;
    if (valid) {
        if (P.rendered) {
            float* o = P.rendered + 3 * pix;
            o[0] = L0; o[1] = L1; o[2] = L2;
        }
        const float* t = P.targets + 3 * pix;
        const float t0 = t[0], t1 = t[1], t2 = t[2];
        d0 = t0 - L0; d1 = t1 - L1; d2 = t2 - L2;
        flame = fmaxf(t0, fmaxf(t1, t2)) > P.thresh;
        if (P.residual) {
            float* o = P.residual + 3 * pix;
            o[0] = flame ? d0 : 0.0f;
            o[1] = flame ? d1 : 0.0f;
            o[2] = flame ? d2 : 0.0f;
        }
        const int* bb = P.bbox + 4 * view;
        if (px >= bb[0] && px <= bb[2] && py >= bb[1] && py <= bb[3]) {
            a0 = d0 * d0; a1 = d1 * d1; a2 = d2 * d2; cnt = 1.0f;
        }
    }
    // the flame ray's number: the tile's offset and its rank in the tile
    __shared__ unsigned wc[kTileThreads / 32];
    __shared__ float red[4][kTileThreads / 32];
    const unsigned m = __ballot_sync(0xffffffffu, flame);
    a0 = warp_sum(a0); a1 = warp_sum(a1); a2 = warp_sum(a2); cnt = warp_sum(cnt);
    if (lane == 0) {
        wc[w] = (unsigned)__popc(m);
        red[0][w] = a0; red[1][w] = a1; red[2][w] = a2; red[3][w] = cnt;
    }
    __syncthreads();
    if (flame) {
        unsigned fid = __ldg(it.tfoff + tile) + (unsigned)__popc(m & ((1u << lane) - 1u));
        for (int i = 0; i < w; ++i) fid += wc[i];
        it.dl[FR_CHK(fid, it.nflame, 8u)] = make_float4(d0, d1, d2, 0.0f);
    }
    if (threadIdx.x < 4) {
        float s = 0.0f;
#pragma unroll
        for (int i = 0; i < kTileThreads / 32; ++i) s += red[threadIdx.x][i];
        P.partials[4 * (long long)tile + threadIdx.x] = s;
    }
}

template <int DT>
__global__ void FR_TAB_FWD_BOUNDS tab_forward_kernel(const __grid_constant__ SingleArgs a, TabIter it)
{
    tab_forward_body<DT>(a.p, it, blockIdx.x);
}

// The same over several problems: CTA b renders tile slot b - tile_start[i]
// of problem i (tile_start ascending, its last entry the total).
template <int DT>
__global__ void FR_TAB_FWD_BOUNDS tab_forward_batch_kernel(const ProbDev* __restrict__ probs,
                                                           const TabIter* __restrict__ its,
                                                           const int* __restrict__ tile_start, int nprob)
{
    const int i = find_problem(tile_start, nprob, blockIdx.x);
    tab_forward_body<DT>(probs[i], its[i], blockIdx.x - (unsigned)__ldg(tile_start + i));
}

// Adjustment and update of the hull's key points: kTabLanes lanes per key
// point sum W times the flame ray's residual over its entries, then one lane
// adds the sum to the record (Eq. 11), clamps it at 0 when asked and stores
// it in the volume's type.  Every key point of the hull is visited each
// iteration (as the update visits every node), entries or not.
#ifndef FR_TAB_LANES
#define FR_TAB_LANES 8
#endif
constexpr int kTabLanes = FR_TAB_LANES;
static_assert(kTabLanes >= 1 && kTabLanes <= 32 && (kTabLanes & (kTabLanes - 1)) == 0, "FR_TAB_LANES: power of 2");
constexpr int kTabAdjThreads = 256;

// stage_next: also write the stored record to it.hs[g], the next iteration's
// staged source (loops without in-scattering, whose source is the volume).
template <int DT>
__device__ __forceinline__ void tab_adjust_body(void* vol, const TabIter& it, int clamp_nonneg, long long nodes,
                                                unsigned blk, bool stage_next)
{
    const unsigned g = (blk * (unsigned)kTabAdjThreads + threadIdx.x) / (unsigned)kTabLanes;
    const unsigned sub = threadIdx.x & (kTabLanes - 1);
    float a0 = 0.0f, a1 = 0.0f, a2 = 0.0f;
#if FR_TAB_ADJ_BULK
    {
        // the warp's key points' entries are one contiguous range
        constexpr unsigned per_warp = 32 / kTabLanes;
        const unsigned g0 = g - (threadIdx.x & 31) / kTabLanes;
        if ((threadIdx.x & 31) == 0 && g0 < it.nhull) {
            const unsigned g1 = min(g0 + per_warp, it.nhull) - 1;
            const unsigned lo = (g0 ? min(__ldg(it.hend + g0 - 1), it.nadj) : 0u) & ~1u;
            // (rounded to whole 16-byte pairs inside the table)
            const unsigned hi = min((min(__ldg(it.hend + g1), it.nadj) + 1u) & ~1u, it.nadj & ~1u);
            if (hi > lo) bulk_prefetch_l2(it.eadj + lo, (hi - lo) * 8u);
        }
    }
#endif
    if (g < it.nhull) {
        const unsigned b = g ? min(__ldg(it.hend + g - 1), it.nadj) : 0u, e = min(__ldg(it.hend + g), it.nadj);
        // kTabAdjUnroll entries per lane at a time, the next group's loaded
        // before this group's residuals are gathered
        unsigned i = b + sub;
        uint2 cur[kTabAdjUnroll];
#pragma unroll
        for (int q = 0; q < kTabAdjUnroll; ++q) {
            const unsigned k = i + q * kTabLanes;
            cur[q] = k < e ? __ldcs(it.eadj + k) : make_uint2(0u, 0u);
        }
        for (; i < e; i += kTabAdjUnroll * kTabLanes) {
            uint2 nxt[kTabAdjUnroll];
#pragma unroll
            for (int q = 0; q < kTabAdjUnroll; ++q) {
                const unsigned k = i + (kTabAdjUnroll + q) * kTabLanes;
                nxt[q] = k < e ? __ldcs(it.eadj + k) : make_uint2(0u, 0u);
            }
            float4 d[kTabAdjUnroll];
#pragma unroll
            for (int q = 0; q < kTabAdjUnroll; ++q)
                d[q] = i + q * kTabLanes < e ? __ldg(it.dl + FR_CHK(cur[q].x, it.nflame, 8u))
                                             : make_float4(0.0f, 0.0f, 0.0f, 0.0f);
#pragma unroll
            for (int q = 0; q < kTabAdjUnroll; ++q) {
                const float W = __uint_as_float(cur[q].y);
                a0 = fmaf(W, d[q].x, a0); a1 = fmaf(W, d[q].y, a1); a2 = fmaf(W, d[q].z, a2);
                cur[q] = nxt[q];
            }
        }
    }
#pragma unroll
    for (int o = kTabLanes / 2; o > 0; o >>= 1) {
        a0 += __shfl_xor_sync(0xffffffffu, a0, o);
        a1 += __shfl_xor_sync(0xffffffffu, a1, o);
        a2 += __shfl_xor_sync(0xffffffffu, a2, o);
    }
    if (g < it.nhull && sub == 0) {
        const long long node = FR_CHK(__ldg(it.hnode + g), nodes, 32u);
        float4 v = load_rgb<DT>(vol, node);
        v.x += a0; v.y += a1; v.z += a2;
        if (clamp_nonneg) {
            v.x = fmaxf(v.x, 0.0f); v.y = fmaxf(v.y, 0.0f); v.z = fmaxf(v.z, 0.0f);
        }
        store_rgb<DT>(vol, node, v);
        if (stage_next) store_rgb<DT>(it.hs, g, v);
    }
}

// CTAs [0, nfin) sum the forward's error partials (finalize_parts_body), the
// rest adjust blocks of key points; the sums are taken first so that they run
// beside the adjustment instead of after it.
template <int DT>
__global__ void __launch_bounds__(kTabAdjThreads) tab_adjust_kernel(void* vol, TabIter it, int clamp_nonneg,
                                                                    long long nodes, FinArgs fin, unsigned nfin)
{
    if (blockIdx.x < nfin) {
        float4* part_sums = reinterpret_cast<float4*>(fin.scratch);
        finalize_parts_body(fin.partials, fin.ntiles, fin.out4, 0, part_sums,
                            reinterpret_cast<unsigned*>(part_sums + kFinParts), fin.rmse3, blockIdx.x, nfin);
        return;
    }
    tab_adjust_body<DT>(vol, it, clamp_nonneg, nodes, blockIdx.x - nfin, false);
}

// The same over several problems: CTA b takes block b - blk_start[i] of
// problem i's key points (blk_start ascending, its last entry the total),
// updates P.vol_rw and stages the next iteration's records.
template <int DT>
__global__ void __launch_bounds__(kTabAdjThreads) tab_adjust_batch_kernel(const ProbDev* __restrict__ probs,
                                                                          const TabIter* __restrict__ its,
                                                                          const int* __restrict__ blk_start, int nprob,
                                                                          int clamp_nonneg)
{
    const int i = find_problem(blk_start, nprob, blockIdx.x);
    const ProbDev& P = probs[i];
    tab_adjust_body<DT>(P.vol_rw, its[i], clamp_nonneg, P.nodes, blockIdx.x - (unsigned)__ldg(blk_start + i), true);
}

}  // namespace

static cudaError_t launch_tab_build(const SingleArgs& a, const TabBuild& b, int dt, int ntiles, int fill,
                                    cudaStream_t s)
{
    if (ntiles <= 0) return cudaSuccess;
    if (dt == DT_F32) tab_build_kernel<DT_F32><<<ntiles, kTileThreads, 0, s>>>(a, b, fill);
    else if (dt == DT_BF16) tab_build_kernel<DT_BF16><<<ntiles, kTileThreads, 0, s>>>(a, b, fill);
    else tab_build_kernel<DT_F16><<<ntiles, kTileThreads, 0, s>>>(a, b, fill);
    return cudaGetLastError();
}

cudaError_t launch_tab_count(const SingleArgs& a, const TabBuild& b, int dt, int ntiles, cudaStream_t s)
{
    return launch_tab_build(a, b, dt, ntiles, 0, s);
}

cudaError_t launch_tab_scans(const TabBuild& b, int ntiles, unsigned long long* bsum, unsigned long long* totals,
                             cudaStream_t s)
{
    const long long nw = (long long)ntiles * (kTileThreads / 32);
    const long long nk = b.order.count();
    cudaError_t e = scan(GetU32{b.wrows}, PutU32{b.woff}, nw, bsum, totals + 0, s);
    if (e == cudaSuccess) e = scan(GetU32{b.tfl}, PutU32{b.tfoff}, ntiles, bsum, totals + 1, s);
    if (e == cudaSuccess)
        e = scan(GetCountOrdered{b.ncnt, b.order}, PutCursorOrdered{b.ncnt, b.order}, nk, bsum, totals + 2, s);
    if (e == cudaSuccess)
        e = scan(GetInHullOrdered{b.tags, b.full, b.order}, PutCompactOrdered{b.hnode, b.order}, nk, bsum,
                 totals + 3, s);
    if (e == cudaSuccess && nk > 0) {
        // hid: each key point's place in the hull's list (nodes outside the hull keep what they held)
        hid_kernel<<<(unsigned)((b.nodes + 255) / 256), 256, 0, s>>>(b.hnode, totals + 3, b.hid);
        e = cudaGetLastError();
    }
    return e;
}

size_t tab_scan_blocks(long long n) { return (size_t)((n + kScanChunk - 1) / kScanChunk); }

cudaError_t launch_tab_fill(const SingleArgs& a, const TabBuild& b, int dt, int ntiles, cudaStream_t s)
{
    return launch_tab_build(a, b, dt, ntiles, 1, s);
}

cudaError_t launch_tab_hend(const unsigned* hnode, const unsigned* cursor, unsigned nh, unsigned* hend, cudaStream_t s)
{
    if (nh == 0) return cudaSuccess;
    hend_kernel<<<(nh + 255) / 256, 256, 0, s>>>(hnode, cursor, nh, hend);
    return cudaGetLastError();
}

#ifndef FR_TAB_SORT
#define FR_TAB_SORT 0
#endif
cudaError_t launch_tab_stage(const void* records, int dt, const TabIter& it, cudaStream_t s)
{
    if (it.nhull == 0) return cudaSuccess;
    const unsigned g = (it.nhull + 255) / 256;
    if (dt == DT_F32)
        stage_kernel<uint4><<<g, 256, 0, s>>>(static_cast<const uint4*>(records), it.hnode, it.nhull,
                                             static_cast<uint4*>(it.hs));
    else
        stage_kernel<uint2><<<g, 256, 0, s>>>(static_cast<const uint2*>(records), it.hnode, it.nhull,
                                             static_cast<uint2*>(it.hs));
    return cudaGetLastError();
}

cudaError_t launch_tab_sort(uint2* eadj, const unsigned* hend, unsigned nh, cudaStream_t s)
{
    if (nh == 0 || !FR_TAB_SORT) return cudaSuccess;
    tab_sort_kernel<<<(nh + kSortWarps - 1) / kSortWarps, 32 * kSortWarps, 0, s>>>(eadj, hend, nh);
    return cudaGetLastError();
}

cudaError_t launch_tab_forward(const SingleArgs& a, const TabIter& it, int dt, int ntiles, cudaStream_t s)
{
    if (ntiles <= 0) return cudaSuccess;
    if (dt == DT_F32) tab_forward_kernel<DT_F32><<<ntiles, kTileThreads, 0, s>>>(a, it);
    else if (dt == DT_BF16) tab_forward_kernel<DT_BF16><<<ntiles, kTileThreads, 0, s>>>(a, it);
    else tab_forward_kernel<DT_F16><<<ntiles, kTileThreads, 0, s>>>(a, it);
    return cudaGetLastError();
}

cudaError_t launch_tab_adjust(void* vol, int dt, long long nodes, const TabIter& it, int clamp_nonneg, cudaStream_t s,
                              const FinArgs* fin)
{
    const FinArgs f = fin ? *fin : FinArgs{};
    const unsigned nfin = fin ? (unsigned)kFinParts : 0u;
    const unsigned g = tab_adjust_blocks(it.nhull) + nfin;
    if (g == 0) return cudaSuccess;
    if (dt == DT_F32) tab_adjust_kernel<DT_F32><<<g, kTabAdjThreads, 0, s>>>(vol, it, clamp_nonneg, nodes, f, nfin);
    else if (dt == DT_BF16)
        tab_adjust_kernel<DT_BF16><<<g, kTabAdjThreads, 0, s>>>(vol, it, clamp_nonneg, nodes, f, nfin);
    else tab_adjust_kernel<DT_F16><<<g, kTabAdjThreads, 0, s>>>(vol, it, clamp_nonneg, nodes, f, nfin);
    return cudaGetLastError();
}

unsigned tab_adjust_blocks(unsigned nh) { return (nh + kTabAdjThreads / kTabLanes - 1) / (kTabAdjThreads / kTabLanes); }

cudaError_t launch_tab_forward_batch(const ProbDev* probs, const TabIter* its, const int* tile_start, int nprob,
                                     int total_tiles, int dt, cudaStream_t s)
{
    if (nprob <= 0 || total_tiles <= 0) return cudaSuccess;
    if (dt == DT_F32) tab_forward_batch_kernel<DT_F32><<<total_tiles, kTileThreads, 0, s>>>(probs, its, tile_start, nprob);
    else if (dt == DT_BF16) tab_forward_batch_kernel<DT_BF16><<<total_tiles, kTileThreads, 0, s>>>(probs, its, tile_start, nprob);
    else tab_forward_batch_kernel<DT_F16><<<total_tiles, kTileThreads, 0, s>>>(probs, its, tile_start, nprob);
    return cudaGetLastError();
}

cudaError_t launch_tab_adjust_batch(const ProbDev* probs, const TabIter* its, const int* blk_start, int nprob,
                                    int total_blocks, int dt, int clamp_nonneg, cudaStream_t s)
{
    if (nprob <= 0 || total_blocks <= 0) return cudaSuccess;
    if (dt == DT_F32)
        tab_adjust_batch_kernel<DT_F32><<<total_blocks, kTabAdjThreads, 0, s>>>(probs, its, blk_start, nprob, clamp_nonneg);
    else if (dt == DT_BF16)
        tab_adjust_batch_kernel<DT_BF16><<<total_blocks, kTabAdjThreads, 0, s>>>(probs, its, blk_start, nprob, clamp_nonneg);
    else
        tab_adjust_batch_kernel<DT_F16><<<total_blocks, kTabAdjThreads, 0, s>>>(probs, its, blk_start, nprob, clamp_nonneg);
    return cudaGetLastError();
}

#ifndef FR_TAB_LPT
#define FR_TAB_LPT 1
#endif
void tab_tile_order(const unsigned* wrows, int ntiles, unsigned* order)
{
    for (int t = 0; t < ntiles; ++t) order[t] = (unsigned)t;
    if (!FR_TAB_LPT) return;
    constexpr int wpt = kTileThreads / 32;
    auto len = [wrows](unsigned t) {
        unsigned m = 0;
        for (int w = 0; w < wpt; ++w) m = std::max(m, wrows[(size_t)t * wpt + w]);
        return m;
    };
    // counting sort by the length, longest first, tile order among equals
    std::vector<unsigned> key(ntiles);
    unsigned kmax = 0;
    for (int t = 0; t < ntiles; ++t) {
        key[t] = len((unsigned)t);
        kmax = std::max(kmax, key[t]);
    }
    std::vector<unsigned> at((size_t)kmax + 2, 0u);
    for (int t = 0; t < ntiles; ++t) ++at[kmax - key[t] + 1];
    for (size_t k = 1; k < at.size(); ++k) at[k] += at[k - 1];
    for (int t = 0; t < ntiles; ++t) order[at[kmax - key[t]]++] = (unsigned)t;
}

cudaError_t check_word_tables(unsigned* word, bool reset)
{
#ifdef FR_CHECKED
    cudaError_t e = cudaMemcpyFromSymbol(word, g_fr_check_word, sizeof(unsigned));
    if (e == cudaSuccess && reset) {
        const unsigned zero = 0;
        e = cudaMemcpyToSymbol(g_fr_check_word, &zero, sizeof(unsigned));
    }
    return e;
#else
    *word = 0;
    (void)reset;
    return cudaSuccess;
#endif
}

}  // namespace frk
