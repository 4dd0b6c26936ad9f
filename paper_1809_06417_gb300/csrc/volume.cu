// volume.cu -- per-node and per-pixel kernels around the ray marches:
//  * apply: V <- V + scale dV (Eq. 11), clamp, re-round to the storage type;
//  * scatter: axis sweeps for the in-scattered radiance (Eq. 5, third term,
//    isotropic phase) and the source records S = q + albedo sigma J;
//  * planck_lut: the colour-temperature table (Sec. 3.3.3);
//  * prepare_targets: flame threshold and flame bounding boxes (Sec. 4.1);
//  * the error of the reconstruction: the volume data error of Sec. 5.1 and the
//    stop criterion's iteration end.
#include "fr_device.cuh"
#include "fr_internal.h"

namespace frk {

// ---------------------------------------------------------------------------
// Apply the accumulated adjustment
// ---------------------------------------------------------------------------

// The update of node i (hull: the hull clear fused into it, see apply_kernel).
template <int DT, int KIND>
__device__ __forceinline__ void apply_node(void* vol, long long i, float* dV, float scale, int with_sigma,
                                           int clamp_nonneg, int zero_dV, const unsigned* __restrict__ hull,
                                           unsigned hull_full)
{
    if (hull && __ldg(hull + i) != hull_full) {
        if constexpr (KIND == KIND_RGB) {
            store_rgb<DT>(vol, i, make_float4(0.0f, 0.0f, 0.0f, 0.0f));
            if (zero_dV) reinterpret_cast<float4*>(dV)[i] = make_float4(0.0f, 0.0f, 0.0f, 0.0f);
        } else {
            store_ts<DT>(vol, i, make_float2(0.0f, 0.0f));
            if (zero_dV) reinterpret_cast<float2*>(dV)[i] = make_float2(0.0f, 0.0f);
        }
        return;
    }
    if constexpr (KIND == KIND_RGB) {
        float4 v = load_rgb<DT>(vol, i);
        float4 d = reinterpret_cast<float4*>(dV)[i];
        v.x = fmaf(scale, d.x, v.x);
        v.y = fmaf(scale, d.y, v.y);
        v.z = fmaf(scale, d.z, v.z);
        if (with_sigma) v.w = fmaf(scale, d.w, v.w);
        if (clamp_nonneg) {
            v.x = fmaxf(v.x, 0.0f); v.y = fmaxf(v.y, 0.0f); v.z = fmaxf(v.z, 0.0f);
            if (with_sigma) v.w = fmaxf(v.w, 0.0f);
        }
        store_rgb<DT>(vol, i, v);
        if (zero_dV) reinterpret_cast<float4*>(dV)[i] = make_float4(0.0f, 0.0f, 0.0f, 0.0f);
    } else {
        float2 v = load_ts<DT>(vol, i);
        float2 d = reinterpret_cast<float2*>(dV)[i];
        v.x = fmaf(scale, d.x, v.x);
        if (with_sigma) v.y = fmaf(scale, d.y, v.y);
        if (clamp_nonneg) {
            v.x = fmaxf(v.x, 0.0f);
            if (with_sigma) v.y = fmaxf(v.y, 0.0f);
        }
        store_ts<DT>(vol, i, v);
        if (zero_dV) reinterpret_cast<float2*>(dV)[i] = make_float2(0.0f, 0.0f);
    }
}

// hull (nullable): records of key points whose tag differs from hull_full
// are set to 0 instead (the hull clear fused into the update).  (A pass over
// the visual hull's bricks only measured slower than this flat one, which
// streams at close to the L2 bandwidth.)
template <int DT, int KIND>
__global__ void __launch_bounds__(256) apply_kernel(void* vol, long long nodes, float* dV, float scale,
                                                    int with_sigma, int clamp_nonneg, int zero_dV,
                                                    const unsigned* __restrict__ hull, unsigned hull_full)
{
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < nodes;
         i += (long long)gridDim.x * blockDim.x)
        apply_node<DT, KIND>(vol, i, dV, scale, with_sigma, clamp_nonneg, zero_dV, hull, hull_full);
}

// Node range [lo, hi] per axis of a NodeBox (false: no flagged brick); the
// same box arithmetic as the marches' BrickSkip::box_range.
__device__ __forceinline__ bool node_range(const NodeBox& B, int nx, int ny, int nz, int lo[3], int hi[3])
{
    const int n[3] = {nx, ny, nz}, nb[3] = {B.nbx, B.nby, B.nbz};
    if (!B.box) {
#pragma unroll
        for (int a = 0; a < 3; ++a) { lo[a] = 0; hi[a] = n[a] - 1; }
        return true;
    }
    if (__ldg(B.box + 3) == 0u) return false;
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        lo[a] = (nb[a] - (int)__ldg(B.box + a)) * kBrick;
        hi[a] = min((int)__ldg(B.box + 3 + a) * kBrick, n[a] - 1);
    }
    return true;
}

// apply_kernel over the nodes of a NodeBox.
template <int DT, int KIND>
__global__ void __launch_bounds__(256) apply_box_kernel(void* vol, int nx, int ny, int nz, float* dV, float scale,
                                                        int with_sigma, int clamp_nonneg, int zero_dV,
                                                        const unsigned* __restrict__ hull, unsigned hull_full,
                                                        NodeBox B)
{
    int lo[3], hi[3];
    if (!node_range(B, nx, ny, nz, lo, hi)) return;
    const unsigned ex = (unsigned)(hi[0] - lo[0] + 1), ey = (unsigned)(hi[1] - lo[1] + 1);
    const unsigned total = ex * ey * (unsigned)(hi[2] - lo[2] + 1);   // volumes hold < 2^31 nodes
    const long long nodes = (long long)nx * ny * nz;   // bounds of the checked build
    (void)nodes;
    for (unsigned t = blockIdx.x * blockDim.x + threadIdx.x; t < total; t += gridDim.x * blockDim.x) {
        const unsigned row = t / ex, x = t - row * ex, z = row / ey, y = row - z * ey;
        const long long i = ((long long)(z + lo[2]) * ny + (y + lo[1])) * nx + (x + lo[0]);
        apply_node<DT, KIND>(vol, FR_CHK(i, nodes, 32u), dV, scale, with_sigma, clamp_nonneg, zero_dV, hull,
                             hull_full);
    }
}

static int grid_for(long long n, int block)
{
    long long g = (n + block - 1) / block;
    const long long cap = 152LL * 16;  // enough resident CTAs for every SM
    return (int)(g < cap ? (g < 1 ? 1 : g) : cap);
}

cudaError_t launch_apply(void* vol, int dt, int kind, long long nodes, float* dV, float scale,
                         int with_sigma, int clamp_nonneg, int zero_dV, cudaStream_t s, const unsigned* hull,
                         unsigned hull_full)
{
    int g = grid_for(nodes, 256);
#define FR_APPLY(D, KD) \
    apply_kernel<D, KD><<<g, 256, 0, s>>>(vol, nodes, dV, scale, with_sigma, clamp_nonneg, zero_dV, hull, hull_full)
    if (kind == KIND_RGB) {
        if (dt == DT_F32) FR_APPLY(DT_F32, KIND_RGB);
        else if (dt == DT_BF16) FR_APPLY(DT_BF16, KIND_RGB);
        else FR_APPLY(DT_F16, KIND_RGB);
    } else {
        if (dt == DT_F32) FR_APPLY(DT_F32, KIND_TEMP);
        else if (dt == DT_BF16) FR_APPLY(DT_BF16, KIND_TEMP);
        else FR_APPLY(DT_F16, KIND_TEMP);
    }
#undef FR_APPLY
    return cudaGetLastError();
}

cudaError_t launch_apply_box(void* vol, int dt, int kind, int nx, int ny, int nz, float* dV, float scale,
                             int with_sigma, int clamp_nonneg, int zero_dV, cudaStream_t s, const unsigned* hull,
                             unsigned hull_full, NodeBox box)
{
    const long long nodes = (long long)nx * ny * nz;
    if (!box.box)
        return launch_apply(vol, dt, kind, nodes, dV, scale, with_sigma, clamp_nonneg, zero_dV, s, hull, hull_full);
    const int g = grid_for(nodes, 256);
#define FR_APPLY(D, KD)                                                                                          \
    apply_box_kernel<D, KD><<<g, 256, 0, s>>>(vol, nx, ny, nz, dV, scale, with_sigma, clamp_nonneg, zero_dV, hull, \
                                              hull_full, box)
    if (kind == KIND_RGB) {
        if (dt == DT_F32) FR_APPLY(DT_F32, KIND_RGB);
        else if (dt == DT_BF16) FR_APPLY(DT_BF16, KIND_RGB);
        else FR_APPLY(DT_F16, KIND_RGB);
    } else {
        if (dt == DT_F32) FR_APPLY(DT_F32, KIND_TEMP);
        else if (dt == DT_BF16) FR_APPLY(DT_BF16, KIND_TEMP);
        else FR_APPLY(DT_F16, KIND_TEMP);
    }
#undef FR_APPLY
    return cudaGetLastError();
}

// Batched apply (paper rule, RGB records): blockIdx.y is the problem; each
// problem's nodes are covered grid-stride.
// FR_BATCH_BOX = 1: with the hull's brick table (the adjustment skipping by
// it), only the nodes of its box (NodeBox): every record outside is zero and
// no adjustment reaches it (the same restriction as the single loop's).
#ifndef FR_BATCH_BOX
#define FR_BATCH_BOX 1
#endif
template <int DT>
__global__ void __launch_bounds__(256) apply_batch_kernel(const ProbDev* __restrict__ probs, int clamp_nonneg)
{
    const ProbDev& P = probs[blockIdx.y];
    void* vol = P.vol_rw;
    float4* dV = reinterpret_cast<float4*>(P.dV);
    int lo[3], hi[3];
    const NodeBox B = FR_BATCH_BOX && P.adj_occ ? NodeBox{P.adj_box, P.nbx, P.nby, P.nbz} : NodeBox{};
    if (!node_range(B, P.nx, P.ny, P.nz, lo, hi)) return;
    const unsigned ex = (unsigned)(hi[0] - lo[0] + 1), ey = (unsigned)(hi[1] - lo[1] + 1);
    const unsigned total = ex * ey * (unsigned)(hi[2] - lo[2] + 1);   // volumes hold < 2^31 nodes
    for (unsigned t = blockIdx.x * blockDim.x + threadIdx.x; t < total; t += gridDim.x * blockDim.x) {
        const unsigned row = t / ex, xo = t - row * ex, zo = row / ey, yo = row - zo * ey;
        const long long i = FR_CHK(((long long)(zo + lo[2]) * P.ny + (yo + lo[1])) * P.nx + (xo + lo[0]), P.nodes, 32u);
        if (P.hull && __ldg(P.hull + i) != P.hull_full) {   // outside the problem's hull: held at 0
            store_rgb<DT>(vol, i, make_float4(0.0f, 0.0f, 0.0f, 0.0f));
            dV[i] = make_float4(0.0f, 0.0f, 0.0f, 0.0f);
            continue;
        }
        float4 v = load_rgb<DT>(vol, i);
        const float4 d = dV[i];
        v.x += d.x; v.y += d.y; v.z += d.z;
        if (clamp_nonneg) { v.x = fmaxf(v.x, 0.0f); v.y = fmaxf(v.y, 0.0f); v.z = fmaxf(v.z, 0.0f); }
        store_rgb<DT>(vol, i, v);
        dV[i] = make_float4(0.0f, 0.0f, 0.0f, 0.0f);
    }
}

cudaError_t launch_apply_batch(const ProbDev* probs, int nprob, int dt, int clamp_nonneg, cudaStream_t s)
{
    const dim3 grid(96, nprob);
    if (dt == DT_F32) apply_batch_kernel<DT_F32><<<grid, 256, 0, s>>>(probs, clamp_nonneg);
    else if (dt == DT_BF16) apply_batch_kernel<DT_BF16><<<grid, 256, 0, s>>>(probs, clamp_nonneg);
    else apply_batch_kernel<DT_F16><<<grid, 256, 0, s>>>(probs, clamp_nonneg);
    return cudaGetLastError();
}

// rmse_all[(p * iters + i) * 3 + c] from each problem's error sums.
__global__ void rmse_batch_kernel(const ProbDev* __restrict__ probs, int nprob, int iters, float* rmse_all)
{
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= nprob * iters) return;
    const int p = t / iters, i = t - p * iters;
    const float* sq = probs[p].sqerr + 4 * i;
    const float cnt = sq[3];
    for (int c = 0; c < 3; ++c) rmse_all[3 * t + c] = cnt > 0.0f ? 255.0f * sqrtf(sq[c] / cnt) : 0.0f;
}

cudaError_t launch_rmse_batch(const ProbDev* probs, int nprob, int iters, float* rmse_all, cudaStream_t s)
{
    const int n = nprob * iters;
    rmse_batch_kernel<<<(n + 127) / 128, 128, 0, s>>>(probs, nprob, iters, rmse_all);
    return cudaGetLastError();
}

// x-pair records: pair i = {record i, record i + 1}, the second copy of the
// last node of a row repeating it (no cell uses it).  One CTA per row.
// Marks, for a non-zero record at node (x, y, z), every brick of kBrick^3 cells
// whose corner records include it (a node on a brick boundary belongs to the
// bricks on both sides).  Stores only ones; the flags are cleared beforehand.
__device__ __forceinline__ void mark_bricks(unsigned char* occ, int x, int y, int z, int nbx, int nby, int nbz)
{
    constexpr int S = kBrickShift, M = kBrick - 1;
    const int bx0 = (x > 0 && (x & M) == 0) ? (x >> S) - 1 : (x >> S);
    const int by0 = (y > 0 && (y & M) == 0) ? (y >> S) - 1 : (y >> S);
    const int bz0 = (z > 0 && (z & M) == 0) ? (z >> S) - 1 : (z >> S);
    for (int bz = bz0; bz <= min(z >> S, nbz - 1); ++bz)
        for (int by = by0; by <= min(y >> S, nby - 1); ++by)
            for (int bx = bx0; bx <= min(x >> S, nbx - 1); ++bx)
                occ[FR_CHK(((long long)bz * nby + by) * nbx + bx, (long long)nbx * nby * nbz, 16u)] = 1;
}


// Merges the box [lo, hi) of brick coordinates seen by the CTA's threads (hi 0:
// none) into the table's box, encoded {nb - lo, hi} per axis and merged with
// atomicMax (the table, box included, is zeroed beforehand).  Every thread of
// the CTA calls it.
__device__ __forceinline__ void merge_box(unsigned char* table, int nbx, int nby, int nbz, const unsigned lo[3],
                                          const unsigned hi[3])
{
    __shared__ unsigned red[6][32];
    const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        const unsigned l = __reduce_min_sync(0xffffffffu, lo[a]), h = __reduce_max_sync(0xffffffffu, hi[a]);
        if (lane == 0) { red[a][w] = l; red[3 + a][w] = h; }
    }
    __syncthreads();
    if (w == 0) {
        const int nw = blockDim.x >> 5;
        unsigned* box = brick_box(table, nbx, nby, nbz);
        const int nbs[3] = {nbx, nby, nbz};
#pragma unroll
        for (int a = 0; a < 3; ++a) {
            const unsigned l = __reduce_min_sync(0xffffffffu, lane < nw ? red[a][lane] : UINT_MAX);
            const unsigned h = __reduce_max_sync(0xffffffffu, lane < nw ? red[3 + a][lane] : 0u);
            if (lane == 0 && h) {
                atomicMax(box + a, (unsigned)nbs[a] - l);
                atomicMax(box + 3 + a, h);
            }
        }
    }
}

// The box of the flagged bricks of a brick table: CTA `part` of `nparts`
// scans its share of the flags and merges its box into the table's with
// atomicMax on the encoded values {nb - lo, hi + 1} (the table, box included,
// is zeroed beforehand).
__device__ __forceinline__ void brick_box_part(unsigned char* table, int nbx, int nby, int nbz, int part,
                                               int nparts)
{
    const int nb = nbx * nby * nbz;
    unsigned lo[3] = {UINT_MAX, UINT_MAX, UINT_MAX}, hi[3] = {0u, 0u, 0u};
    for (int b = part * blockDim.x + threadIdx.x; b < nb; b += nparts * blockDim.x) {
        if (!table[b]) continue;
        const unsigned c[3] = {(unsigned)(b % nbx), (unsigned)((b / nbx) % nby), (unsigned)(b / (nbx * nby))};
#pragma unroll
        for (int a = 0; a < 3; ++a) {
            lo[a] = min(lo[a], c[a]);
            hi[a] = max(hi[a], c[a] + 1u);
        }
    }
    merge_box(table, nbx, nby, nbz, lo, hi);
}

constexpr int kBoxParts = 16;   // CTAs per brick table

__global__ void __launch_bounds__(256) brick_box_kernel(unsigned char* table, int nbx, int nby, int nbz)
{
    brick_box_part(table, nbx, nby, nbz, blockIdx.x, gridDim.x);
}

// Batched forms, one problem per blockIdx.y (reset, box) or per CTA (box).
__global__ void __launch_bounds__(256) brick_reset_batch_kernel(const ProbDev* __restrict__ probs)
{
    const ProbDev& P = probs[blockIdx.y];
    if (!P.occ) return;
    unsigned char* t = const_cast<unsigned char*>(P.occ);
    const size_t n = brick_table_bytes(P.nx, P.ny, P.nz);
    for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x)
        t[i] = 0;
}

__global__ void __launch_bounds__(256) brick_box_batch_kernel(const ProbDev* __restrict__ probs)
{
    const ProbDev& P = probs[blockIdx.y];
    if (!P.occ) return;
    brick_box_part(const_cast<unsigned char*>(P.occ), P.nbx, P.nby, P.nbz, blockIdx.x, gridDim.x);
}

cudaError_t launch_brick_reset_batch(const ProbDev* probs, int nprob, cudaStream_t s)
{
    brick_reset_batch_kernel<<<dim3(8, nprob), 256, 0, s>>>(probs);
    return cudaGetLastError();
}

cudaError_t launch_brick_box_batch(const ProbDev* probs, int nprob, cudaStream_t s)
{
    brick_box_batch_kernel<<<dim3(kBoxParts, nprob), 256, 0, s>>>(probs);
    return cudaGetLastError();
}

static cudaError_t launch_brick_box(unsigned char* table, int nx, int ny, int nz, cudaStream_t s)
{
    brick_box_kernel<<<kBoxParts, 256, 0, s>>>(table, bricks_along(nx), bricks_along(ny), bricks_along(nz));
    return cudaGetLastError();
}

// A brick table whose flagged-off bricks hold zero records (flags nullable:
// none): the nodes of those bricks are read by no forward sample.
struct KeepBricks {
    const unsigned char* flags;
    int nx, ny, nbx, nby, nbz;
};

// Nodes owned by brick (bx, by, bz): [B b, B b + B) along each axis, the last
// brick along an axis owning the nodes up to n - 1 as well (B = kBrick).  The
// bricks that hold an owned node are the brick itself and its lower
// neighbours, so when none of those is flagged in a table whose flagged-off
// bricks hold zero records, the owned nodes need no pass.
struct OwnedNodes {
    int x0, y0, z0, ex, ey, ez;
    bool active;
};

__device__ __forceinline__ OwnedNodes owned_nodes(const KeepBricks& K, int nz, int b)
{
    OwnedNodes o;
    const int bx = b % K.nbx, r = b / K.nbx, by = r % K.nby, bz = r / K.nby;
    o.active = false;
    for (int cz = max(bz - 1, 0); cz <= bz; ++cz)
        for (int cy = max(by - 1, 0); cy <= by; ++cy)
            for (int cx = max(bx - 1, 0); cx <= bx; ++cx)
                o.active |= __ldg(K.flags + FR_CHK(((long long)cz * K.nby + cy) * K.nbx + cx,
                                                   (long long)K.nbx * K.nby * K.nbz, 40u)) != 0;
    o.x0 = bx * kBrick; o.y0 = by * kBrick; o.z0 = bz * kBrick;
    o.ex = bx == K.nbx - 1 ? K.nx - o.x0 : kBrick;
    o.ey = by == K.nby - 1 ? K.ny - o.y0 : kBrick;
    o.ez = bz == K.nbz - 1 ? nz - o.z0 : kBrick;
    return o;
}

// Pair i = {record i, record of its +x neighbour} (itself from x = x_last
// on: the grid's last x, or the last x of the box the records are known in)
// of node (x, y, z), and the brick marks of the non-zero records.
template <int DT, int KIND>
__device__ __forceinline__ void pack_node(const void* src, void* dst, long long i, int x, int y, int z, int x_last,
                                          unsigned char* occ, int nbx, int nby, int nbz)
{
    const long long j = x < x_last ? i + 1 : i;
    if constexpr (KIND == KIND_RGB) {
        bool nonzero;
        if constexpr (DT == DT_F32) {
            const float4* s4 = reinterpret_cast<const float4*>(src);
            float4* d4 = reinterpret_cast<float4*>(dst);
            const float4 a = __ldg(s4 + i);
            d4[2 * i] = a;
            d4[2 * i + 1] = __ldg(s4 + j);
            nonzero = a.x != 0.0f || a.y != 0.0f || a.z != 0.0f || a.w != 0.0f;
        } else {
            const uint2* s2 = reinterpret_cast<const uint2*>(src);
            const uint2 a = __ldg(s2 + i), b = __ldg(s2 + j);
            reinterpret_cast<uint4*>(dst)[i] = make_uint4(a.x, a.y, b.x, b.y);
            nonzero = ((a.x | a.y) & 0x7fff7fffu) != 0u;   // +0 and -0 both read as empty
        }
        if (occ && nonzero) mark_bricks(occ, x, y, z, nbx, nby, nbz);
    } else {
        if constexpr (DT == DT_F32) {
            const float2* s2 = reinterpret_cast<const float2*>(src);
            const float2 a = __ldg(s2 + i), b = __ldg(s2 + j);
            reinterpret_cast<float4*>(dst)[i] = make_float4(a.x, a.y, b.x, b.y);
        } else {
            const unsigned* s1 = reinterpret_cast<const unsigned*>(src);
            reinterpret_cast<uint2*>(dst)[i] = make_uint2(__ldg(s1 + i), __ldg(s1 + j));
        }
    }
}

// Flat over the nodes (every thread busy whatever nx is).
template <int DT, int KIND>
__global__ void __launch_bounds__(256) pair_pack_kernel(const void* src, void* dst, long long nodes, int nx, int ny,
                                                        unsigned char* occ, int nbx, int nby, int nbz)
{
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < nodes;
         i += (long long)gridDim.x * blockDim.x) {
        // node coordinates in 32-bit arithmetic (volumes hold < 2^31 nodes)
        const unsigned row = (unsigned)i / (unsigned)nx;
        const int x = (int)((unsigned)i - row * (unsigned)nx);
        const unsigned z = row / (unsigned)ny;
        const int y = (int)(row - z * (unsigned)ny);
        pack_node<DT, KIND>(src, dst, i, x, y, (int)z, nx - 1, occ, nbx, nby, nbz);
    }
}

// Over the owned nodes of the active bricks of `keep` only, one warp per brick
// (a node of an inactive brick is read by no forward sample).  With a
// NodeBox, the records are known inside it only (the sweeps computed no more;
// every record outside it is zero): nodes outside are left out, and the pair
// of the box's last x node repeats that node, zero like its neighbour -- the
// same pairs and brick marks as over the whole grid, for the cells the
// forward can evaluate.
template <int DT, int KIND>
__global__ void __launch_bounds__(256) pair_pack_bricks_kernel(const void* src, void* dst, int nz, unsigned char* occ,
                                                               KeepBricks keep, NodeBox B)
{
    const int b = (int)((blockIdx.x * (unsigned)blockDim.x + threadIdx.x) >> 5), lane = threadIdx.x & 31;
    if (b >= keep.nbx * keep.nby * keep.nbz) return;
    const OwnedNodes o = owned_nodes(keep, nz, b);
    if (!o.active) return;
    int lo[3], hi[3];
    if (!node_range(B, keep.nx, keep.ny, nz, lo, hi)) return;
    const int x_last = min(keep.nx - 1, hi[0]);
    const int exy = o.ex * o.ey, cnt = exy * o.ez;
    for (int t = lane; t < cnt; t += 32) {
        const int dz = t / exy, r = t - dz * exy, dy = r / o.ex, dx = r - dy * o.ex;
        const int x = o.x0 + dx, y = o.y0 + dy, z = o.z0 + dz;
        if (x < lo[0] || x > hi[0] || y < lo[1] || y > hi[1] || z < lo[2] || z > hi[2]) continue;
        const long long i = ((long long)z * keep.ny + y) * keep.nx + x;
        pack_node<DT, KIND>(src, dst, i, x, y, z, x_last, occ, keep.nbx, keep.nby, keep.nbz);
    }
}

// Batched form: blockIdx.y is the problem, its volume vol_rw packed into pairs.
template <int DT>
__global__ void __launch_bounds__(256) pair_pack_batch_kernel(const ProbDev* __restrict__ probs)
{
    const ProbDev& P = probs[blockIdx.y];
    const int nx = P.nx;
    const void* src = P.vol_rw;
    void* dst = const_cast<void*>(P.pairs);
    unsigned char* occ = const_cast<unsigned char*>(P.occ);   // brick flags (cleared beforehand), or null
    // with the hull's brick table, the rows and nodes of its box only (see
    // apply_batch_kernel): the records outside are zero, so are their pairs
    // and marks, and the forward evaluates no cell there; the pair of the
    // box's last x node repeats that node, zero like its neighbour
    int lo[3], hi[3];
    const NodeBox B = FR_BATCH_BOX && P.adj_occ ? NodeBox{P.adj_box, P.nbx, P.nby, P.nbz} : NodeBox{};
    if (!node_range(B, P.nx, P.ny, P.nz, lo, hi)) return;
    const int ey = hi[1] - lo[1] + 1, x_last = min(nx - 1, hi[0]);
    const long long rows = (long long)ey * (hi[2] - lo[2] + 1);
    for (long long rb = blockIdx.x; rb < rows; rb += gridDim.x) {
        const int yy = lo[1] + (int)(rb % ey), zz = lo[2] + (int)(rb / ey);
        const long long row = (long long)zz * P.ny + yy, r0 = row * nx;
        for (int x = lo[0] + threadIdx.x; x <= hi[0]; x += blockDim.x) {
            const long long i = FR_CHK(r0 + x, P.nodes, 32u), j = x < x_last ? i + 1 : i;
            bool nonzero;
            if constexpr (DT == DT_F32) {
                const float4* s4 = reinterpret_cast<const float4*>(src);
                float4* d4 = reinterpret_cast<float4*>(dst);
                const float4 a = s4[i];
                d4[2 * i] = a;
                d4[2 * i + 1] = s4[j];
                nonzero = a.x != 0.0f || a.y != 0.0f || a.z != 0.0f || a.w != 0.0f;
            } else {
                const uint2* s2 = reinterpret_cast<const uint2*>(src);
                const uint2 a = s2[i], b = s2[j];
                reinterpret_cast<uint4*>(dst)[i] = make_uint4(a.x, a.y, b.x, b.y);
                nonzero = ((a.x | a.y) & 0x7fff7fffu) != 0u;
            }
            if (occ && nonzero) mark_bricks(occ, x, (int)(row % P.ny), (int)(row / P.ny), P.nbx, P.nby, P.nbz);
        }
    }
}

cudaError_t launch_pair_pack_batch(const ProbDev* probs, int nprob, int dt, cudaStream_t s)
{
    const dim3 grid(256, nprob);
    if (dt == DT_F32) pair_pack_batch_kernel<DT_F32><<<grid, 256, 0, s>>>(probs);
    else if (dt == DT_BF16) pair_pack_batch_kernel<DT_BF16><<<grid, 256, 0, s>>>(probs);
    else pair_pack_batch_kernel<DT_F16><<<grid, 256, 0, s>>>(probs);
    return cudaGetLastError();
}

cudaError_t launch_pair_pack(const void* src, void* dst, int dt, int kind, int nx, int ny, int nz,
                             unsigned char* occ, cudaStream_t s, const unsigned char* keep, NodeBox box)
{
    const long long nodes = (long long)nx * ny * nz;
    const int g = grid_for(nodes, 256);
    const int nbx = (nx - 2) / kBrick + 1, nby = (ny - 2) / kBrick + 1, nbz = (nz - 2) / kBrick + 1;
    if (occ) {
        cudaError_t e = cudaMemsetAsync(occ, 0, brick_table_bytes(nx, ny, nz), s);
        if (e != cudaSuccess) return e;
    }
    const KeepBricks KB{keep, nx, ny, nbx, nby, nbz};
    const unsigned gb = (unsigned)(((long long)nbx * nby * nbz * 32 + 255) / 256);
#define FR_PACK(D, K)                                                                        \
    if (keep) pair_pack_bricks_kernel<D, K><<<gb, 256, 0, s>>>(src, dst, nz, occ, KB, box); \
    else pair_pack_kernel<D, K><<<g, 256, 0, s>>>(src, dst, nodes, nx, ny, occ, nbx, nby, nbz)
    if (kind == KIND_RGB) {
        if (dt == DT_F32) FR_PACK(DT_F32, KIND_RGB);
        else if (dt == DT_BF16) FR_PACK(DT_BF16, KIND_RGB);
        else FR_PACK(DT_F16, KIND_RGB);
    } else {
        if (dt == DT_F32) FR_PACK(DT_F32, KIND_TEMP);
        else if (dt == DT_BF16) FR_PACK(DT_BF16, KIND_TEMP);
        else FR_PACK(DT_F16, KIND_TEMP);
    }
#undef FR_PACK
    if (occ && !keep) {
        cudaError_t e = cudaGetLastError();
        if (e != cudaSuccess) return e;
        return launch_brick_box(occ, nx, ny, nz, s);
    }
    return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// In-scattering: J = (1/6) sum over the six axis directions of the emitted
// radiance arriving along grid lines; each unit segment between adjacent nodes
// is sampled at its midpoint (the mean of its two end records).
// ---------------------------------------------------------------------------

// The recurrence along a line, L(i) = L(i-1) e_i + c_i with e_i = exp(-s) and
// c_i = q (1 - exp(-s)) / s for the unit segment into node i (s, q the means of
// its two end records), is an affine map per segment, so a line is scanned in
// chunks: each chunk composes its segments' maps (forward and backward), the
// chunks of a line combine their maps through shared memory, and each chunk
// then walks its nodes again from its incoming radiance.  A CTA holds kSweepLines lines
// (threadIdx.x, neighbouring lines: coalesced for the y and z sweeps) times
// kSweepChunks chunks (threadIdx.y).  The x sweep initialises J, the z sweep
// (LAST) finishes it and writes the source records S = q + albedo sigma J.
// (Staging a CTA's 32 lines in shared memory, one coalesced load pass and two
// CTAs per SM, measured 15% slower than holding each chunk in registers.)
// (Testing the visual hull's brick table first, so that chunks in bricks
// known to be zero skip their loads, measured 15% slower: the flag load adds
// a dependent round trip to every chunk of these latency-bound sweeps.)
// 16 lines per CTA (256 threads with 16 chunks): the same arithmetic per line
// as 32 and twice the CTAs, measured 6% faster over the hull's box at 128^3
// (0.048 against 0.051 ms for the three sweeps); 16 lines of 32 chunks 0.049,
// 32 lines of 32 chunks 0.053 ms.
#ifndef FR_SWEEP_LINES
#define FR_SWEEP_LINES 16
#endif
constexpr int kSweepLines = FR_SWEEP_LINES;
// 16 chunks per line (8 nodes each at 128^3): twice the threads of 8 chunks
// and half the serial walk, measured 10% faster; 32 chunks gained nothing more.
#ifndef FR_SWEEP_CHUNKS
#define FR_SWEEP_CHUNKS 16
#endif
constexpr int kSweepChunks = FR_SWEEP_CHUNKS;

struct Seg {
    float e, c0, c1, c2;
};

__device__ __forceinline__ bool nonzero_record(float4 r)
{
    return r.x != 0.0f || r.y != 0.0f || r.z != 0.0f || r.w != 0.0f;
}

template <int DT>
__device__ __forceinline__ Seg seg_between(float4 a, float4 b)
{
    const float sig = 0.5f * (a.w + b.w);
    const float e = __expf(-sig);
    const float beta = seg_weight(sig, 1.0f, e);
    return Seg{e, 0.5f * (a.x + b.x) * beta, 0.5f * (a.y + b.y) * beta, 0.5f * (a.z + b.z) * beta};
}

// L6 (nullable): store each direction's radiance there (nodes x 6 float4)
// instead of accumulating J and writing the source.
template <int DT, int AXIS, bool LAST>
__global__ void __launch_bounds__(kSweepLines * kSweepChunks) sweep_kernel(const void* em, const float* albedo,
                                                                            float* J, void* out, int nx, int ny,
                                                                            int nz, float4* L6, bool skip_empty)
{
    __shared__ float4 fwd[kSweepChunks][kSweepLines];   // {E, C0, C1, C2} of each chunk, forward
    __shared__ float4 bwd[kSweepChunks][kSweepLines];   // and backward
    const int n_line = AXIS == 0 ? nx : (AXIS == 1 ? ny : nz);
    const long long lines = AXIS == 0 ? (long long)ny * nz : (AXIS == 1 ? (long long)nx * nz : (long long)nx * ny);
    const long long line = blockIdx.x * (long long)kSweepLines + threadIdx.x;
    const int ch = threadIdx.y;
    const bool live = line < lines;
    long long start = 0, stride = 1;
    if (live) {
        if constexpr (AXIS == 0) {
            start = line * nx;                       // line = z * ny + y
            stride = 1;
        } else if constexpr (AXIS == 1) {
            const long long z = line / nx, x = line - z * nx;
            start = z * (long long)nx * ny + x;
            stride = nx;
        } else {
            start = line;                            // line = y * nx + x
            stride = (long long)nx * ny;
        }
    }
    const int m = (n_line + kSweepChunks - 1) / kSweepChunks;
    const int s0 = min(ch * m, n_line), s1 = min(s0 + m, n_line);   // nodes [s0, s1) of this chunk

    // phase 1: compose the forward map of the segments into s0..s1-1 and the
    // backward map of the segments into s1-1..s0
    float Ef = 1.0f, F0 = 0.0f, F1 = 0.0f, F2 = 0.0f;
    float Eb = 1.0f, B0 = 0.0f, B1 = 0.0f, B2 = 0.0f;
    bool occupied = false;   // some record of the chunk's nodes is non-zero
    if (live && s1 > s0) {
        const int lo = max(s0 - 1, 0), hi = min(s1, n_line - 1);
        float4 prev = load_rgb<DT>(em, start + lo * stride);
        if (lo == s0) occupied = nonzero_record(prev);
        for (int i = lo + 1; i <= hi; ++i) {
            const float4 cur = load_rgb<DT>(em, start + i * stride);
            if (i < s1) occupied |= nonzero_record(cur);
            const Seg g = seg_between<DT>(prev, cur);
            if (i >= s0 && i < s1) {   // forward segment into node i
                F0 = fmaf(F0, g.e, g.c0); F1 = fmaf(F1, g.e, g.c1); F2 = fmaf(F2, g.e, g.c2);
                Ef *= g.e;
            }
            if (i - 1 >= s0 && i - 1 < s1) {   // backward segment into node i - 1
                B0 = fmaf(Eb, g.c0, B0); B1 = fmaf(Eb, g.c1, B1); B2 = fmaf(Eb, g.c2, B2);
                Eb *= g.e;
            }
            prev = cur;
        }
    }
    fwd[ch][threadIdx.x] = make_float4(Ef, F0, F1, F2);
    bwd[ch][threadIdx.x] = make_float4(Eb, B0, B1, B2);
    __syncthreads();
    if (!live || s1 <= s0) return;
    if (skip_empty && !occupied) {
        // every record of the chunk is zero: no extinction, so J at its nodes
        // is never used (S = q + albedo sigma J = 0 there); the light crossing
        // it is carried by the chunk maps.  Only the stores the next steps
        // read are made: zero directional radiances, or the zero source.
        for (int i = s0; i < s1; ++i) {
            const long long node = FR_CHK(start + i * stride, (long long)nx * ny * nz, 32u);
            if (L6) {
                L6[6 * node + 2 * AXIS] = make_float4(0.0f, 0.0f, 0.0f, 0.0f);
                L6[6 * node + 2 * AXIS + 1] = make_float4(0.0f, 0.0f, 0.0f, 0.0f);
            } else if constexpr (LAST) {
                store_rgb<DT>(out, node, make_float4(0.0f, 0.0f, 0.0f, 0.0f));
            }
        }
        return;
    }

    // phase 2: radiance arriving at the chunk from either side
    float lf0 = 0.0f, lf1 = 0.0f, lf2 = 0.0f;
    for (int c = 0; c < ch; ++c) {
        const float4 f = fwd[c][threadIdx.x];
        lf0 = fmaf(lf0, f.x, f.y); lf1 = fmaf(lf1, f.x, f.z); lf2 = fmaf(lf2, f.x, f.w);
    }
    float lb0 = 0.0f, lb1 = 0.0f, lb2 = 0.0f;
    for (int c = kSweepChunks - 1; c > ch; --c) {
        const float4 b = bwd[c][threadIdx.x];
        lb0 = fmaf(lb0, b.x, b.y); lb1 = fmaf(lb1, b.x, b.z); lb2 = fmaf(lb2, b.x, b.w);
    }

    // phase 3: walk the chunk forward (J += L_forward / 6) ...
    const float sixth = 1.0f / 6.0f;
    float4* J4 = reinterpret_cast<float4*>(J);
    {
        float4 prev = load_rgb<DT>(em, start + max(s0 - 1, 0) * stride);
        for (int i = s0; i < s1; ++i) {
            const long long node = FR_CHK(start + i * stride, (long long)nx * ny * nz, 32u);
            const float4 cur = load_rgb<DT>(em, node);
            if (i > 0) {
                const Seg g = seg_between<DT>(prev, cur);
                lf0 = fmaf(lf0, g.e, g.c0); lf1 = fmaf(lf1, g.e, g.c1); lf2 = fmaf(lf2, g.e, g.c2);
            }
            prev = cur;
            if (L6) {
                L6[6 * node + 2 * AXIS] = make_float4(lf0, lf1, lf2, 0.0f);
                continue;
            }
            float4 j;
            if constexpr (AXIS == 0) {
                j = make_float4(lf0 * sixth, lf1 * sixth, lf2 * sixth, 0.0f);
            } else {
                j = J4[node];
                j.x = fmaf(lf0, sixth, j.x); j.y = fmaf(lf1, sixth, j.y); j.z = fmaf(lf2, sixth, j.z);
            }
            J4[node] = j;
        }
    }
    // ... and backward (J += L_backward / 6; the z sweep then writes S)
    {
        float4 next = load_rgb<DT>(em, start + min(s1, n_line - 1) * stride);
        for (int i = s1 - 1; i >= s0; --i) {
            const long long node = FR_CHK(start + i * stride, (long long)nx * ny * nz, 32u);
            const float4 cur = load_rgb<DT>(em, node);
            if (i < n_line - 1) {
                const Seg g = seg_between<DT>(cur, next);
                lb0 = fmaf(lb0, g.e, g.c0); lb1 = fmaf(lb1, g.e, g.c1); lb2 = fmaf(lb2, g.e, g.c2);
            }
            next = cur;
            if (L6) {
                L6[6 * node + 2 * AXIS + 1] = make_float4(lb0, lb1, lb2, 0.0f);
                continue;
            }
            float4 j = J4[node];
            j.x = fmaf(lb0, sixth, j.x); j.y = fmaf(lb1, sixth, j.y); j.z = fmaf(lb2, sixth, j.z);
            if constexpr (LAST) {
                const float as = __ldg(albedo + node) * cur.w;
                store_rgb<DT>(out, node, make_float4(fmaf(as, j.x, cur.x), fmaf(as, j.y, cur.y),
                                                     fmaf(as, j.z, cur.z), cur.w));
            }
            J4[node] = j;
        }
    }
}

// A source record in its storage form (the bits store_rgb writes) and
// whether it is non-zero as stored (+0 and -0 read as empty, as in the pack).
template <int DT>
__device__ __forceinline__ bool stored_form(float4 v, float4& f, uint2& u)
{
    if constexpr (DT == DT_F32) {
        f = v;
        return v.x != 0.0f || v.y != 0.0f || v.z != 0.0f || v.w != 0.0f;
    } else {
        if constexpr (DT == DT_BF16) {
            __nv_bfloat162 a = __floats2bfloat162_rn(v.x, v.y), b = __floats2bfloat162_rn(v.z, v.w);
            u.x = *reinterpret_cast<uint32_t*>(&a);
            u.y = *reinterpret_cast<uint32_t*>(&b);
        } else {
            __half2 a = __floats2half2_rn(v.x, v.y), b = __floats2half2_rn(v.z, v.w);
            u.x = *reinterpret_cast<uint32_t*>(&a);
            u.y = *reinterpret_cast<uint32_t*>(&b);
        }
        return ((u.x | u.y) & 0x7fff7fffu) != 0u;
    }
}

template <int DT>
__device__ __forceinline__ void put_stored(void* dst, long long i, const float4& f, const uint2& u)
{
    if constexpr (DT == DT_F32) reinterpret_cast<float4*>(dst)[i] = f;
    else reinterpret_cast<uint2*>(dst)[i] = u;
}

// Source record of node `node` at (x, y, z) written to `out` and, with pk, to
// the two x-pairs that hold it (its own first half, the -x neighbour's second
// half inside the box, its own second half on the box's last x), with the
// brick marks of a non-zero record.
template <int DT>
__device__ __forceinline__ void put_source(void* out, long long node, float4 v, const PackOut& pk, int x, int y, int z,
                                           int x_lo, int x_last, int nbx, int nby, int nbz)
{
    float4 f;
    uint2 u;
    const bool nz = stored_form<DT>(v, f, u);
    put_stored<DT>(out, node, f, u);
    if (pk.pairs) {
        put_stored<DT>(pk.pairs, 2 * node, f, u);
        if (x > x_lo) put_stored<DT>(pk.pairs, 2 * node - 1, f, u);
        if (x == x_last) put_stored<DT>(pk.pairs, 2 * node + 1, f, u);
        if (nz && pk.occ) mark_bricks(pk.occ, x, y, z, nbx, nby, nbz);
    }
}

// The y / z sweep with a chunk of at most CM nodes held in registers: the
// chunk's records (and its nodes' J, albedo) are loaded together at the start,
// where the kernel above reloads them in three dependent walks; J is stored
// once per node.  The arithmetic and its order are the same, so the results
// are bitwise equal.  rec[0] is node max(s0 - 1, 0), rec[1 + q] node s0 + q,
// rec[cnt + 1] node min(s1, n - 1); segment j joins rec[j] and rec[j + 1] and
// leads into node s0 + j.
//
// With a NodeBox, only the lines through the box run, over the box's nodes:
// every record outside it is zero, so the light reaching the box along a line
// is zero and the segment into its first node (from a zero record) is part of
// the first chunk, as without the box.
template <int DT, int AXIS, bool LAST, int CM>
__global__ void __launch_bounds__(kSweepLines * kSweepChunks) sweep_reg_kernel(const void* em, const float* albedo,
                                                                                float* J, void* out, int nx, int ny,
                                                                                int nz, bool skip_empty, NodeBox B,
                                                                                PackOut pk)
{
    static_assert(!LAST || AXIS == 2, "the source (and its pairs) is written by the z sweep");
    __shared__ float4 fwd[kSweepChunks][kSweepLines];
    __shared__ float4 bwd[kSweepChunks][kSweepLines];
    const int n_line = AXIS == 1 ? ny : nz;
    const long long lines = AXIS == 1 ? (long long)nx * nz : (long long)nx * ny;
    const long long line = blockIdx.x * (long long)kSweepLines + threadIdx.x;
    const int ch = threadIdx.y;
    int lo[3], hi[3];
    bool live = line < lines && node_range(B, nx, ny, nz, lo, hi);
    long long start = 0, stride = 1;
    int lx = 0, lc = 0;   // the line's x and its other coordinate (z for y lines, y for z lines)
    if (live) {
        const int c = (int)(line / nx), x = (int)(line - (long long)c * nx);
        lx = x;
        lc = c;
        const int ca = AXIS == 1 ? 2 : 1;
        live = x >= lo[0] && x <= hi[0] && c >= lo[ca] && c <= hi[ca];
        if constexpr (AXIS == 1) {
            start = (long long)c * nx * ny + x;      // line = z * nx + x
            stride = nx;
        } else {
            start = line;                            // line = y * nx + x
            stride = (long long)nx * ny;
        }
    }
    const long long nodes = (long long)nx * ny * nz;   // bounds of the checked build
    (void)nodes;
    const int alo = live ? lo[AXIS] : 0, ahi = live ? hi[AXIS] : -1;   // the nodes [alo, ahi] of the line
    const int m = (ahi - alo + 1 + kSweepChunks - 1) / kSweepChunks;
    const int s0 = min(alo + ch * m, ahi + 1), s1 = min(s0 + m, ahi + 1), cnt = s1 - s0;   // cnt <= CM
    float4 rec[CM + 2];
    float Ef = 1.0f, F0 = 0.0f, F1 = 0.0f, F2 = 0.0f;
    float Eb = 1.0f, B0 = 0.0f, B1 = 0.0f, B2 = 0.0f;
    bool occupied = false;
    float3 jv[CM];   // J of the chunk's nodes (earlier sweeps), then J + L_forward / 6
    float alb[CM];
    if (live && cnt > 0) {
#pragma unroll
        for (int j = 0; j < CM + 2; ++j) {
            if (j <= cnt + 1) {
                const int i = j == 0 ? max(s0 - 1, 0) : (j <= cnt ? s0 + j - 1 : min(s1, n_line - 1));
                rec[j] = load_rgb<DT>(em, FR_CHK(start + i * stride, nodes, 35u));
            }
        }
#pragma unroll
        for (int q = 0; q < CM; ++q)
            if (q < cnt) occupied |= nonzero_record(rec[q + 1]);
        if (!skip_empty || occupied) {
            float4* J4 = reinterpret_cast<float4*>(J);
#pragma unroll
            for (int q = 0; q < CM; ++q) {
                if (q < cnt) {
                    const long long node = start + (s0 + q) * stride;
                    const float4 t = J4[node];
                    jv[q] = make_float3(t.x, t.y, t.z);
                    if constexpr (LAST) alb[q] = __ldg(albedo + node);
                }
            }
        }
        // phase 1: the chunk's forward and backward maps
#pragma unroll
        for (int j = 0; j <= CM; ++j) {
            const int i = s0 + j;
            if (j <= cnt && i >= 1 && i <= n_line - 1) {
                const Seg g = seg_between<DT>(rec[j], rec[j + 1]);
                if (j < cnt) {
                    F0 = fmaf(F0, g.e, g.c0); F1 = fmaf(F1, g.e, g.c1); F2 = fmaf(F2, g.e, g.c2);
                    Ef *= g.e;
                }
                if (j >= 1) {
                    B0 = fmaf(Eb, g.c0, B0); B1 = fmaf(Eb, g.c1, B1); B2 = fmaf(Eb, g.c2, B2);
                    Eb *= g.e;
                }
            }
        }
    }
    fwd[ch][threadIdx.x] = make_float4(Ef, F0, F1, F2);
    bwd[ch][threadIdx.x] = make_float4(Eb, B0, B1, B2);
    __syncthreads();
    if (!live || cnt <= 0) return;
    const int x_last = min(nx - 1, hi[0]);   // (pk: lines through the box only, so lo/hi are set)
    if (skip_empty && !occupied) {
        if constexpr (LAST) {
            for (int q = 0; q < cnt; ++q)
                put_source<DT>(out, FR_CHK(start + (s0 + q) * stride, nodes, 36u), make_float4(0.0f, 0.0f, 0.0f, 0.0f),
                               pk, lx, lc, s0 + q, lo[0], x_last, B.nbx, B.nby, B.nbz);
        }
        return;
    }
    // phase 2: radiance arriving at the chunk from either side
    float lf0 = 0.0f, lf1 = 0.0f, lf2 = 0.0f;
    for (int c = 0; c < ch; ++c) {
        const float4 f = fwd[c][threadIdx.x];
        lf0 = fmaf(lf0, f.x, f.y); lf1 = fmaf(lf1, f.x, f.z); lf2 = fmaf(lf2, f.x, f.w);
    }
    float lb0 = 0.0f, lb1 = 0.0f, lb2 = 0.0f;
    for (int c = kSweepChunks - 1; c > ch; --c) {
        const float4 b = bwd[c][threadIdx.x];
        lb0 = fmaf(lb0, b.x, b.y); lb1 = fmaf(lb1, b.x, b.z); lb2 = fmaf(lb2, b.x, b.w);
    }
    // phase 3: forward walk (J += L_forward / 6, in registers) ...
    const float sixth = 1.0f / 6.0f;
#pragma unroll
    for (int q = 0; q < CM; ++q) {
        if (q < cnt) {
            if (s0 + q > 0) {
                const Seg g = seg_between<DT>(rec[q], rec[q + 1]);
                lf0 = fmaf(lf0, g.e, g.c0); lf1 = fmaf(lf1, g.e, g.c1); lf2 = fmaf(lf2, g.e, g.c2);
            }
            jv[q].x = fmaf(lf0, sixth, jv[q].x); jv[q].y = fmaf(lf1, sixth, jv[q].y);
            jv[q].z = fmaf(lf2, sixth, jv[q].z);
        }
    }
    // ... and backward walk (J += L_backward / 6; stored, or the source written)
    float4* J4 = reinterpret_cast<float4*>(J);
#pragma unroll
    for (int q = CM - 1; q >= 0; --q) {
        if (q < cnt) {
            const int i = s0 + q;
            if (i < n_line - 1) {
                const Seg g = seg_between<DT>(rec[q + 1], rec[q + 2]);
                lb0 = fmaf(lb0, g.e, g.c0); lb1 = fmaf(lb1, g.e, g.c1); lb2 = fmaf(lb2, g.e, g.c2);
            }
            const float jx = fmaf(lb0, sixth, jv[q].x), jy = fmaf(lb1, sixth, jv[q].y), jz = fmaf(lb2, sixth, jv[q].z);
            const long long node = FR_CHK(start + i * stride, nodes, 37u);
            if constexpr (LAST) {
                const float4 cur = rec[q + 1];
                const float as = alb[q] * cur.w;
                put_source<DT>(out, node, make_float4(fmaf(as, jx, cur.x), fmaf(as, jy, cur.y), fmaf(as, jz, cur.z), cur.w),
                               pk, lx, lc, i, lo[0], x_last, B.nbx, B.nby, B.nbz);
                if (!skip_empty) J4[node] = make_float4(jx, jy, jz, 0.0f);
            } else {
                J4[node] = make_float4(jx, jy, jz, 0.0f);
            }
        }
    }
}

// The x sweep with one warp per grid line: lane l owns the l-th of 32 chunks
// of consecutive nodes, so a warp's loads walk along one row of memory.  The
// chunks' affine maps are combined with warp shuffles: an inclusive prefix
// (forward maps, composed first-then-next) and an inclusive suffix (backward
// maps).  It initialises J (the first sweep).
template <int DT>
__global__ void __launch_bounds__(256) sweep_x_kernel(const void* em, float* J, int nx, int ny, int nz, float4* L6,
                                                      bool skip_empty)
{
    const unsigned FULL = 0xffffffffu;
    const int lane = threadIdx.x & 31;
    const long long line = blockIdx.x * (long long)(blockDim.x >> 5) + (threadIdx.x >> 5);
    if (line >= (long long)ny * nz) return;   // whole warps leave together
    const long long start = line * nx;
    const int m = (nx + 31) / 32;
    const int s0 = min(lane * m, nx), s1 = min(s0 + m, nx);
    float Ef = 1.0f, F0 = 0.0f, F1 = 0.0f, F2 = 0.0f;
    float Eb = 1.0f, B0 = 0.0f, B1 = 0.0f, B2 = 0.0f;
    bool occupied = false;   // some record of the chunk's nodes is non-zero
    if (s1 > s0) {
        const int lo = max(s0 - 1, 0), hi = min(s1, nx - 1);
        float4 prev = load_rgb<DT>(em, start + lo);
        if (lo == s0) occupied = nonzero_record(prev);
        for (int i = lo + 1; i <= hi; ++i) {
            const float4 cur = load_rgb<DT>(em, start + i);
            if (i < s1) occupied |= nonzero_record(cur);
            const Seg g = seg_between<DT>(prev, cur);
            if (i >= s0 && i < s1) {
                F0 = fmaf(F0, g.e, g.c0); F1 = fmaf(F1, g.e, g.c1); F2 = fmaf(F2, g.e, g.c2);
                Ef *= g.e;
            }
            if (i - 1 >= s0 && i - 1 < s1) {
                B0 = fmaf(Eb, g.c0, B0); B1 = fmaf(Eb, g.c1, B1); B2 = fmaf(Eb, g.c2, B2);
                Eb *= g.e;
            }
            prev = cur;
        }
    }
    // inclusive prefix of the forward maps: (earlier) then (mine)
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const float e = __shfl_up_sync(FULL, Ef, o), c0 = __shfl_up_sync(FULL, F0, o);
        const float c1 = __shfl_up_sync(FULL, F1, o), c2 = __shfl_up_sync(FULL, F2, o);
        if (lane >= o) {
            F0 = fmaf(c0, Ef, F0); F1 = fmaf(c1, Ef, F1); F2 = fmaf(c2, Ef, F2);
            Ef *= e;
        }
    }
    // inclusive suffix of the backward maps: (mine) applied after (later)
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const float e = __shfl_down_sync(FULL, Eb, o), c0 = __shfl_down_sync(FULL, B0, o);
        const float c1 = __shfl_down_sync(FULL, B1, o), c2 = __shfl_down_sync(FULL, B2, o);
        if (lane + o < 32) {
            B0 = fmaf(c0, Eb, B0); B1 = fmaf(c1, Eb, B1); B2 = fmaf(c2, Eb, B2);
            Eb *= e;
        }
    }
    // radiance arriving at the chunk: line start / end carry nothing
    float lf0 = __shfl_up_sync(FULL, F0, 1), lf1 = __shfl_up_sync(FULL, F1, 1), lf2 = __shfl_up_sync(FULL, F2, 1);
    float lb0 = __shfl_down_sync(FULL, B0, 1), lb1 = __shfl_down_sync(FULL, B1, 1), lb2 = __shfl_down_sync(FULL, B2, 1);
    if (lane == 0) { lf0 = lf1 = lf2 = 0.0f; }
    if (lane == 31) { lb0 = lb1 = lb2 = 0.0f; }
    if (s1 <= s0) return;
    const float sixth = 1.0f / 6.0f;
    float4* J4 = reinterpret_cast<float4*>(J);
    if (skip_empty && !occupied) {
        // an empty chunk (see sweep_kernel): J = 0 so that later sweeps add to
        // a defined value, zero directional radiances in L6 mode
        for (int i = s0; i < s1; ++i) {
            if (L6) {
                L6[6 * (start + i)] = make_float4(0.0f, 0.0f, 0.0f, 0.0f);
                L6[6 * (start + i) + 1] = make_float4(0.0f, 0.0f, 0.0f, 0.0f);
            } else {
                J4[start + i] = make_float4(0.0f, 0.0f, 0.0f, 0.0f);
            }
        }
        return;
    }
    {
        float4 prev = load_rgb<DT>(em, start + max(s0 - 1, 0));
        for (int i = s0; i < s1; ++i) {
            const float4 cur = load_rgb<DT>(em, start + i);
            if (i > 0) {
                const Seg g = seg_between<DT>(prev, cur);
                lf0 = fmaf(lf0, g.e, g.c0); lf1 = fmaf(lf1, g.e, g.c1); lf2 = fmaf(lf2, g.e, g.c2);
            }
            prev = cur;
            if (L6) L6[6 * (start + i)] = make_float4(lf0, lf1, lf2, 0.0f);
            else J4[start + i] = make_float4(lf0 * sixth, lf1 * sixth, lf2 * sixth, 0.0f);
        }
    }
    {
        float4 next = load_rgb<DT>(em, start + min(s1, nx - 1));
        for (int i = s1 - 1; i >= s0; --i) {
            const float4 cur = load_rgb<DT>(em, start + i);
            if (i < nx - 1) {
                const Seg g = seg_between<DT>(cur, next);
                lb0 = fmaf(lb0, g.e, g.c0); lb1 = fmaf(lb1, g.e, g.c1); lb2 = fmaf(lb2, g.e, g.c2);
            }
            next = cur;
            if (L6) {
                L6[6 * (start + i) + 1] = make_float4(lb0, lb1, lb2, 0.0f);
                continue;
            }
            float4 j = J4[start + i];
            j.x = fmaf(lb0, sixth, j.x); j.y = fmaf(lb1, sixth, j.y); j.z = fmaf(lb2, sixth, j.z);
            J4[start + i] = j;
        }
    }
}

// The x sweep with a chunk of at most CM nodes held in registers (see
// sweep_reg_kernel; the same arithmetic as sweep_x_kernel in the same order).
// With a NodeBox, the lines through the box over its nodes (as in sweep_reg_kernel).
template <int DT, int CM>
__global__ void __launch_bounds__(256) sweep_x_reg_kernel(const void* em, float* J, int nx, int ny, int nz,
                                                          bool skip_empty, NodeBox B)
{
    const unsigned FULL = 0xffffffffu;
    const int lane = threadIdx.x & 31;
    const long long line = blockIdx.x * (long long)(blockDim.x >> 5) + (threadIdx.x >> 5);
    if (line >= (long long)ny * nz) return;   // whole warps leave together
    int lo[3], hi[3];
    if (!node_range(B, nx, ny, nz, lo, hi)) return;
    {
        const int z = (int)(line / ny), y = (int)(line - (long long)z * ny);   // line = z * ny + y
        if (y < lo[1] || y > hi[1] || z < lo[2] || z > hi[2]) return;
    }
    const long long start = line * nx;
    const long long nodes = (long long)nx * ny * nz;   // bounds of the checked build
    (void)nodes;
    const int m = (hi[0] - lo[0] + 1 + 31) / 32;
    const int s0 = min(lo[0] + lane * m, hi[0] + 1), s1 = min(s0 + m, hi[0] + 1), cnt = s1 - s0;   // cnt <= CM
    float4 rec[CM + 2];
    float Ef = 1.0f, F0 = 0.0f, F1 = 0.0f, F2 = 0.0f;
    float Eb = 1.0f, B0 = 0.0f, B1 = 0.0f, B2 = 0.0f;
    bool occupied = false;
    if (cnt > 0) {
#pragma unroll
        for (int j = 0; j < CM + 2; ++j) {
            if (j <= cnt + 1) {
                const int i = j == 0 ? max(s0 - 1, 0) : (j <= cnt ? s0 + j - 1 : min(s1, nx - 1));
                rec[j] = load_rgb<DT>(em, FR_CHK(start + i, nodes, 38u));
            }
        }
#pragma unroll
        for (int q = 0; q < CM; ++q)
            if (q < cnt) occupied |= nonzero_record(rec[q + 1]);
#pragma unroll
        for (int j = 0; j <= CM; ++j) {
            const int i = s0 + j;
            if (j <= cnt && i >= 1 && i <= nx - 1) {
                const Seg g = seg_between<DT>(rec[j], rec[j + 1]);
                if (j < cnt) {
                    F0 = fmaf(F0, g.e, g.c0); F1 = fmaf(F1, g.e, g.c1); F2 = fmaf(F2, g.e, g.c2);
                    Ef *= g.e;
                }
                if (j >= 1) {
                    B0 = fmaf(Eb, g.c0, B0); B1 = fmaf(Eb, g.c1, B1); B2 = fmaf(Eb, g.c2, B2);
                    Eb *= g.e;
                }
            }
        }
    }
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const float e = __shfl_up_sync(FULL, Ef, o), c0 = __shfl_up_sync(FULL, F0, o);
        const float c1 = __shfl_up_sync(FULL, F1, o), c2 = __shfl_up_sync(FULL, F2, o);
        if (lane >= o) {
            F0 = fmaf(c0, Ef, F0); F1 = fmaf(c1, Ef, F1); F2 = fmaf(c2, Ef, F2);
            Ef *= e;
        }
    }
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const float e = __shfl_down_sync(FULL, Eb, o), c0 = __shfl_down_sync(FULL, B0, o);
        const float c1 = __shfl_down_sync(FULL, B1, o), c2 = __shfl_down_sync(FULL, B2, o);
        if (lane + o < 32) {
            B0 = fmaf(c0, Eb, B0); B1 = fmaf(c1, Eb, B1); B2 = fmaf(c2, Eb, B2);
            Eb *= e;
        }
    }
    float lf0 = __shfl_up_sync(FULL, F0, 1), lf1 = __shfl_up_sync(FULL, F1, 1), lf2 = __shfl_up_sync(FULL, F2, 1);
    float lb0 = __shfl_down_sync(FULL, B0, 1), lb1 = __shfl_down_sync(FULL, B1, 1), lb2 = __shfl_down_sync(FULL, B2, 1);
    if (lane == 0) { lf0 = lf1 = lf2 = 0.0f; }
    if (lane == 31) { lb0 = lb1 = lb2 = 0.0f; }
    if (cnt <= 0) return;
    const float sixth = 1.0f / 6.0f;
    float4* J4 = reinterpret_cast<float4*>(J);
    if (skip_empty && !occupied) {
        for (int q = 0; q < cnt; ++q) J4[start + s0 + q] = make_float4(0.0f, 0.0f, 0.0f, 0.0f);
        return;
    }
    float3 jv[CM];
#pragma unroll
    for (int q = 0; q < CM; ++q) {
        if (q < cnt) {
            if (s0 + q > 0) {
                const Seg g = seg_between<DT>(rec[q], rec[q + 1]);
                lf0 = fmaf(lf0, g.e, g.c0); lf1 = fmaf(lf1, g.e, g.c1); lf2 = fmaf(lf2, g.e, g.c2);
            }
            jv[q] = make_float3(lf0 * sixth, lf1 * sixth, lf2 * sixth);
        }
    }
#pragma unroll
    for (int q = CM - 1; q >= 0; --q) {
        if (q < cnt) {
            const int i = s0 + q;
            if (i < nx - 1) {
                const Seg g = seg_between<DT>(rec[q + 1], rec[q + 2]);
                lb0 = fmaf(lb0, g.e, g.c0); lb1 = fmaf(lb1, g.e, g.c1); lb2 = fmaf(lb2, g.e, g.c2);
            }
            J4[FR_CHK(start + i, nodes, 39u)] =
                make_float4(fmaf(lb0, sixth, jv[q].x), fmaf(lb1, sixth, jv[q].y), fmaf(lb2, sixth, jv[q].z), 0.0f);
        }
    }
}

// Chunks of up to FR_SWEEP_REG_MAX (4 or 8; 0: none) nodes run the
// register-held sweep kernels.
#ifndef FR_SWEEP_REG_MAX
#define FR_SWEEP_REG_MAX 8
#endif

template <int DT, int AXIS, bool LAST>
static cudaError_t launch_sweep_yz(int m, unsigned grid, const void* em, const float* albedo, float* J, void* out,
                                   int nx, int ny, int nz, cudaStream_t s, bool skip_empty, NodeBox box, PackOut pk)
{
    const dim3 B(kSweepLines, kSweepChunks);
    if (FR_SWEEP_REG_MAX >= 4 && m <= 4)
        sweep_reg_kernel<DT, AXIS, LAST, 4><<<grid, B, 0, s>>>(em, albedo, J, out, nx, ny, nz, skip_empty, box, pk);
    else if (FR_SWEEP_REG_MAX >= 8 && m <= 8)
        sweep_reg_kernel<DT, AXIS, LAST, 8><<<grid, B, 0, s>>>(em, albedo, J, out, nx, ny, nz, skip_empty, box, pk);
    else
        sweep_kernel<DT, AXIS, LAST><<<grid, B, 0, s>>>(em, albedo, J, out, nx, ny, nz, nullptr, skip_empty);
    return cudaSuccess;
}

bool sweeps_take_box(int nx, int ny, int nz)
{
    const int cm = FR_SWEEP_REG_MAX >= 8 ? 8 : FR_SWEEP_REG_MAX;
    return (nx + 31) / 32 <= cm && (ny + kSweepChunks - 1) / kSweepChunks <= cm &&
           (nz + kSweepChunks - 1) / kSweepChunks <= cm;
}

template <int DT>
static cudaError_t launch_sweeps(const void* em, const float* albedo, float* J, void* out, int nx, int ny, int nz,
                                 cudaStream_t s, bool skip_empty, NodeBox box, PackOut pk)
{
    const long long lx = (long long)ny * nz, ly = (long long)nx * nz, lz = (long long)nx * ny;
    const unsigned gxw = (unsigned)((lx + 7) / 8);  // one warp per x line, 8 warps per CTA
    const unsigned gy = (unsigned)((ly + kSweepLines - 1) / kSweepLines);
    const unsigned gz = (unsigned)((lz + kSweepLines - 1) / kSweepLines);
    const int mx = (nx + 31) / 32;
    const int my = (ny + kSweepChunks - 1) / kSweepChunks, mz = (nz + kSweepChunks - 1) / kSweepChunks;
    // the box applies when every sweep runs register-held chunks (it is a
    // restriction of work, never needed for the result); so do the pairs
    if (!sweeps_take_box(nx, ny, nz)) {
        if (pk.pairs) return cudaErrorInvalidValue;
        box = NodeBox{};
    }
    if (pk.pairs && !box.box) return cudaErrorInvalidValue;
    if (FR_SWEEP_REG_MAX >= 4 && mx <= 4)
        sweep_x_reg_kernel<DT, 4><<<gxw, 256, 0, s>>>(em, J, nx, ny, nz, skip_empty, box);
    else if (FR_SWEEP_REG_MAX >= 8 && mx <= 8)
        sweep_x_reg_kernel<DT, 8><<<gxw, 256, 0, s>>>(em, J, nx, ny, nz, skip_empty, box);
    else
        sweep_x_kernel<DT><<<gxw, 256, 0, s>>>(em, J, nx, ny, nz, nullptr, skip_empty);
    cudaError_t e = launch_sweep_yz<DT, 1, false>(my, gy, em, albedo, J, out, nx, ny, nz, s, skip_empty, box, PackOut{});
    if (e != cudaSuccess) return e;
    return launch_sweep_yz<DT, 2, true>(mz, gz, em, albedo, J, out, nx, ny, nz, s, skip_empty, box, pk);
}

cudaError_t launch_scatter_source(const void* emission, int dt_in, const float* albedo, float* J,
                                  void* out, int dt_out, int nx, int ny, int nz, cudaStream_t s, bool skip_empty,
                                  NodeBox box, PackOut pk)
{
    if (dt_in != dt_out) return cudaErrorInvalidValue;
    cudaError_t e;
    if (dt_in == DT_F32) e = launch_sweeps<DT_F32>(emission, albedo, J, out, nx, ny, nz, s, skip_empty, box, pk);
    else if (dt_in == DT_BF16) e = launch_sweeps<DT_BF16>(emission, albedo, J, out, nx, ny, nz, s, skip_empty, box, pk);
    else e = launch_sweeps<DT_F16>(emission, albedo, J, out, nx, ny, nz, s, skip_empty, box, pk);
    if (e != cudaSuccess) return e;
    return cudaGetLastError();
}

cudaError_t launch_scatter_L6(const void* emission, int dt, float* L6, int nx, int ny, int nz, cudaStream_t s,
                              bool skip_empty)
{
    const long long lx = (long long)ny * nz, ly = (long long)nx * nz, lz = (long long)nx * ny;
    const unsigned gxw = (unsigned)((lx + 7) / 8);
    const unsigned gy = (unsigned)((ly + kSweepLines - 1) / kSweepLines);
    const unsigned gz = (unsigned)((lz + kSweepLines - 1) / kSweepLines);
    const dim3 B(kSweepLines, kSweepChunks);
    float4* L = reinterpret_cast<float4*>(L6);
#define FR_SWEEPS6(D)                                                                            \
    sweep_x_kernel<D><<<gxw, 256, 0, s>>>(emission, nullptr, nx, ny, nz, L, skip_empty);                    \
    sweep_kernel<D, 1, false><<<gy, B, 0, s>>>(emission, nullptr, nullptr, nullptr, nx, ny, nz, L, skip_empty); \
    sweep_kernel<D, 2, false><<<gz, B, 0, s>>>(emission, nullptr, nullptr, nullptr, nx, ny, nz, L, skip_empty)
    if (dt == DT_F32) { FR_SWEEPS6(DT_F32); }
    else if (dt == DT_BF16) { FR_SWEEPS6(DT_BF16); }
    else { FR_SWEEPS6(DT_F16); }
#undef FR_SWEEPS6
    return cudaGetLastError();
}

// Source records towards one view: S = q + albedo sigma sum_d w_d L_d (Eq. 9
// phase weights), sigma unchanged.
template <int DT>
__global__ void __launch_bounds__(256) source_hg_kernel(const void* em, const float* __restrict__ albedo,
                                                        const float4* __restrict__ L6, HgWeights w, void* out,
                                                        long long nodes)
{
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < nodes;
         i += (long long)gridDim.x * blockDim.x) {
        const float4 r = load_rgb<DT>(em, i);
        float s0 = 0.0f, s1 = 0.0f, s2 = 0.0f;
#pragma unroll
        for (int d = 0; d < 6; ++d) {
            const float4 l = __ldg(L6 + 6 * i + d);
            s0 = fmaf(w.w[d], l.x, s0); s1 = fmaf(w.w[d], l.y, s1); s2 = fmaf(w.w[d], l.z, s2);
        }
        const float as = __ldg(albedo + i) * r.w;
        store_rgb<DT>(out, i, make_float4(fmaf(as, s0, r.x), fmaf(as, s1, r.y), fmaf(as, s2, r.z), r.w));
    }
}

cudaError_t launch_source_hg(const void* emission, int dt, const float* albedo, const float* L6, HgWeights w,
                             void* out, long long nodes, cudaStream_t s)
{
    const int g = grid_for(nodes, 256);
    const float4* L = reinterpret_cast<const float4*>(L6);
    if (dt == DT_F32) source_hg_kernel<DT_F32><<<g, 256, 0, s>>>(emission, albedo, L, w, out, nodes);
    else if (dt == DT_BF16) source_hg_kernel<DT_BF16><<<g, 256, 0, s>>>(emission, albedo, L, w, out, nodes);
    else source_hg_kernel<DT_F16><<<g, 256, 0, s>>>(emission, albedo, L, w, out, nodes);
    return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// Colour-temperature table: Planck's law (Sec. 3.3.3) integrated against three
// Gaussian channel responses by the trapezoid rule, 380-780 nm in 1 nm steps,
// normalised so that green(2000 K) = 1.
// ---------------------------------------------------------------------------

__device__ float planck_um(float lambda_um, float T)
{
    // second radiation constant h c / k in micrometre kelvin; the first
    // constant cancels in the normalisation
    const float c2 = 14387.768775f;
    float l2 = lambda_um * lambda_um;
    return 1.0f / (l2 * l2 * lambda_um * expm1f(c2 / (lambda_um * T)));
}

__device__ void channel_sums(float T, float out[3])
{
    const float mu[3] = {600.0f, 540.0f, 460.0f};
    float acc[3] = {0.0f, 0.0f, 0.0f};
    for (int i = 0; i <= 400; ++i) {
        float lam = 380.0f + (float)i;
        float w = (i == 0 || i == 400) ? 0.5f : 1.0f;
        float b = w * planck_um(lam * 1e-3f, T);
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            float u = (lam - mu[c]) * (1.0f / 40.0f);
            acc[c] = fmaf(b, expf(-0.5f * u * u), acc[c]);
        }
    }
    out[0] = acc[0]; out[1] = acc[1]; out[2] = acc[2];
}

__global__ void planck_lut_kernel(float t_min, float t_max, int m, float4* lut)
{
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= m) return;
    float norm[3], v[3];
    channel_sums(2000.0f, norm);
    float T = t_min + (t_max - t_min) * (float)i / (float)(m - 1);
    channel_sums(T, v);
    float s = 1.0f / norm[1];
    lut[i] = make_float4(v[0] * s, v[1] * s, v[2] * s, 0.0f);
}

cudaError_t launch_planck_lut(float t_min, float t_max, int m, float* lut, cudaStream_t s)
{
    planck_lut_kernel<<<(m + 127) / 128, 128, 0, s>>>(t_min, t_max, m, reinterpret_cast<float4*>(lut));
    return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// Target pre-processing (Sec. 4.1)
// ---------------------------------------------------------------------------

__global__ void bbox_init_kernel(int* bbox, int ncam, int W, int H)
{
    int v = blockIdx.x * blockDim.x + threadIdx.x;
    if (v < ncam) {
        bbox[4 * v + 0] = W; bbox[4 * v + 1] = H; bbox[4 * v + 2] = -1; bbox[4 * v + 3] = -1;
    }
}

// One thread per pixel; grid.y = view.  Rows of the launch are image rows so
// a warp never straddles two views.
__global__ void __launch_bounds__(256) prepare_kernel(float* targets, int W, int H, float thresh, int* bbox)
{
    const int v = blockIdx.y;
    const long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    const bool in = i < (long long)W * H;
    int px = 0, py = 0;
    bool flame = false;
    if (in) {
        py = (int)(i / W);
        px = (int)(i - (long long)py * W);
        float* t = targets + 3 * ((long long)v * W * H + i);
        flame = fmaxf(t[0], fmaxf(t[1], t[2])) > thresh;
        if (!flame) { t[0] = 0.0f; t[1] = 0.0f; t[2] = 0.0f; }
    }
    const unsigned any = __ballot_sync(0xffffffffu, flame);
    if (!any) return;
    int x0 = __reduce_min_sync(0xffffffffu, flame ? px : INT_MAX);
    int y0 = __reduce_min_sync(0xffffffffu, flame ? py : INT_MAX);
    int x1 = __reduce_max_sync(0xffffffffu, flame ? px : -1);
    int y1 = __reduce_max_sync(0xffffffffu, flame ? py : -1);
    if ((threadIdx.x & 31) == 0) {
        atomicMin(bbox + 4 * v + 0, x0);
        atomicMin(bbox + 4 * v + 1, y0);
        atomicMax(bbox + 4 * v + 2, x1);
        atomicMax(bbox + 4 * v + 3, y1);
    }
}

cudaError_t launch_prepare_targets(float* targets, int ncam, int H, int W, float thresh, int* bbox,
                                   cudaStream_t s)
{
    bbox_init_kernel<<<(ncam + 31) / 32, 32, 0, s>>>(bbox, ncam, W, H);
    long long npx = (long long)W * H;
    dim3 grid((unsigned)((npx + 255) / 256), ncam);
    prepare_kernel<<<grid, 256, 0, s>>>(targets, W, H, thresh, bbox);
    return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// Visual hull (Sec. 4.3.1, Algorithm 1)
// ---------------------------------------------------------------------------

// Summed-area table of the flame mask: sat[v][y+1][x+1] = number of flame
// pixels in [0, x] x [0, y] of view v (row 0 and column 0 are zero).
// Summed-area table of each view's flame mask, (H + 1) x (W + 1) per view:
// entry (y, x) counts the flame pixels in image rows < y and columns < x.
// Pass 1: row prefix sums, one warp per table row, 32 columns per step with a
// shuffle scan.
__global__ void __launch_bounds__(256) sat_rows_kernel(const float* targets, int ncam, int W, int H, float thresh,
                                                       unsigned* sat)
{
    const unsigned FULL = 0xffffffffu;
    const int r = (int)((blockIdx.x * (unsigned)blockDim.x + threadIdx.x) >> 5), lane = threadIdx.x & 31;
    if (r >= ncam * (H + 1)) return;   // whole warps leave together
    const int v = r / (H + 1), y = r - v * (H + 1);
    unsigned* row = sat + (size_t)r * (W + 1);
    if (lane == 0) row[0] = 0;
    unsigned carry = 0;
    for (int x0 = 0; x0 < W; x0 += 32) {
        const int x = x0 + lane;
        unsigned f = 0;
        if (y > 0 && x < W) {
            const float* t = targets + 3 * (((size_t)v * H + (y - 1)) * W + x);
            f = fmaxf(t[0], fmaxf(t[1], t[2])) > thresh ? 1u : 0u;
        }
        unsigned incl = f;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const unsigned n = __shfl_up_sync(FULL, incl, o);
            if (lane >= o) incl += n;
        }
        if (x < W) row[x + 1] = carry + incl;
        carry += __shfl_sync(FULL, incl, 31);
    }
}

// Pass 2: column prefix sums.  A CTA takes 32 neighbouring columns of one view
// (threadIdx.x) in kSatChunks row chunks (threadIdx.y): each chunk sums its
// rows, the chunks' sums are combined in shared memory, then each chunk
// rewrites its rows from its offset.
constexpr int kSatChunks = 16;

__global__ void __launch_bounds__(32 * kSatChunks) sat_cols_kernel(int ncam, int W, int H, unsigned* sat)
{
    __shared__ unsigned part[kSatChunks][32];
    const int tiles = (W + 1 + 31) / 32;
    const int v = blockIdx.x / tiles, tile = blockIdx.x - v * tiles;
    const int x = tile * 32 + threadIdx.x, ch = threadIdx.y;
    const bool live = v < ncam && x <= W;
    const int rows = H + 1, m = (rows + kSatChunks - 1) / kSatChunks;
    const int y0 = min(ch * m, rows), y1 = min(y0 + m, rows);
    const size_t w1 = (size_t)W + 1;
    unsigned* base = sat + (size_t)v * rows * w1 + x;
    unsigned sum = 0;
    if (live)
        for (int y = y0; y < y1; ++y) sum += base[y * w1];
    part[ch][threadIdx.x] = sum;
    __syncthreads();
    if (!live) return;
    unsigned acc = 0;
    for (int c = 0; c < ch; ++c) acc += part[c][threadIdx.x];
    for (int y = y0; y < y1; ++y) {
        acc += base[y * w1];
        base[y * w1] = acc;
    }
}

__device__ __forceinline__ float dot3_rn(float x, float y, float z, const float r[3])
{
    return __fadd_rn(__fadd_rn(__fmul_rn(x, r[0]), __fmul_rn(y, r[1])), __fmul_rn(z, r[2]));
}

// `cams` carries o (voxel units), r, u, f, tx, ty, W, H.
struct HullCams {
    CamDev c[kMaxViews];
};

// Pixel coordinates of lattice point (gx, gy, gz) in view c (float32, the
// rounding of each step fixed); false when it is not in front of the camera.
__device__ __forceinline__ bool hull_project(const CamDev& c, int gx, int gy, int gz, float& uu, float& vv)
{
    const float X = __fsub_rn((float)gx, c.o[0]), Y = __fsub_rn((float)gy, c.o[1]), Z = __fsub_rn((float)gz, c.o[2]);
    const float xc = dot3_rn(X, Y, Z, c.r), yc = dot3_rn(X, Y, Z, c.u), zc = dot3_rn(X, Y, Z, c.f);
    if (!(zc > 0.0f)) return false;
    const float hw = 0.5f * (float)c.W, hh = 0.5f * (float)c.H;
    uu = __fsub_rn(__fmul_rn(__fadd_rn(__fdiv_rn(__fdiv_rn(xc, zc), c.tx), 1.0f), hw), 0.5f);
    vv = __fsub_rn(__fmul_rn(__fsub_rn(1.0f, __fdiv_rn(__fdiv_rn(yc, zc), c.ty)), hh), 0.5f);
    return true;
}

// One thread per node, a CTA per tile of kHullTX x kHullTY x kHullTZ nodes.
// Node (i, j, k)'s box has its corners on the lattice points {max(i-1, 0),
// min(i+1, n-1)} per axis, so the tile's nodes share the corners of a
// (kHullTX + 2) x (kHullTY + 2) x (kHullTZ + 2) lattice block: per view the CTA
// projects that block once into shared memory (about 2.3 projections per node
// instead of 8), and each node takes the bounding rectangle of its 8 corners'
// projections and counts the flame pixels in it with 4 table reads.
constexpr int kHullTX = 8, kHullTY = 8, kHullTZ = 4;
constexpr int kHullLX = kHullTX + 2, kHullLY = kHullTY + 2, kHullLZ = kHullTZ + 2;
constexpr int kHullLattice = kHullLX * kHullLY * kHullLZ;

__global__ void __launch_bounds__(kHullTX * kHullTY * kHullTZ) hull_kernel(const __grid_constant__ HullCams cams,
                                                                          int ncam, int nx, int ny, int nz,
                                                                          const unsigned* __restrict__ sat,
                                                                          unsigned* __restrict__ tags)
{
    __shared__ float2 proj[kHullLattice];
    __shared__ unsigned char front[kHullLattice];
    const int tiles_x = (nx + kHullTX - 1) / kHullTX, tiles_y = (ny + kHullTY - 1) / kHullTY;
    const int tb = blockIdx.x, tile_x = tb % tiles_x, tr = tb / tiles_x, tile_y = tr % tiles_y,
              tile_z = tr / tiles_y;
    const int x0 = tile_x * kHullTX, y0 = tile_y * kHullTY, z0 = tile_z * kHullTZ;
    const int t = threadIdx.x;
    const int i = x0 + t % kHullTX, j = y0 + (t / kHullTX) % kHullTY, k = z0 + t / (kHullTX * kHullTY);
    const bool live = i < nx && j < ny && k < nz;
    // lattice indices of the node's box corners within the block (origin x0 - 1, y0 - 1, z0 - 1)
    const int lo[3] = {max(i - 1, 0) - (x0 - 1), max(j - 1, 0) - (y0 - 1), max(k - 1, 0) - (z0 - 1)};
    const int hi[3] = {min(i + 1, nx - 1) - (x0 - 1), min(j + 1, ny - 1) - (y0 - 1), min(k + 1, nz - 1) - (z0 - 1)};
    unsigned tag = 0;
    size_t sat_off = 0;
    for (int v = 0; v < ncam; ++v) {
        const CamDev& c = cams.c[v];
        const int W = c.W, H = c.H;
        for (int p = t; p < kHullLattice; p += blockDim.x) {
            const int pi = p % kHullLX, pr = p / kHullLX, pj = pr % kHullLY, pk = pr / kHullLY;
            float uu = 0.0f, vv = 0.0f;
            front[p] = hull_project(c, x0 - 1 + pi, y0 - 1 + pj, z0 - 1 + pk, uu, vv) ? 1 : 0;
            proj[p] = make_float2(uu, vv);
        }
        __syncthreads();
        if (live) {
            float umin = INFINITY, umax = -INFINITY, vmin = INFINITY, vmax = -INFINITY;
            bool behind = false;
#pragma unroll
            for (int b = 0; b < 8; ++b) {
                const int q = (((b & 4) ? hi[2] : lo[2]) * kHullLY + ((b & 2) ? hi[1] : lo[1])) * kHullLX +
                              ((b & 1) ? hi[0] : lo[0]);
                behind |= front[q] == 0;
                const float2 uv = proj[q];
                umin = fminf(umin, uv.x); umax = fmaxf(umax, uv.x);
                vmin = fminf(vmin, uv.y); vmax = fmaxf(vmax, uv.y);
            }
            int x0p = 0, x1p = W - 1, y0p = 0, y1p = H - 1;
            if (!behind) {
                const float cx0 = ceilf(umin), cx1 = floorf(umax), cy0 = ceilf(vmin), cy1 = floorf(vmax);
                x0p = cx0 > 0.0f ? (cx0 < (float)W ? (int)cx0 : W) : 0;
                x1p = cx1 < (float)(W - 1) ? (cx1 >= -1.0f ? (int)cx1 : -1) : W - 1;
                y0p = cy0 > 0.0f ? (cy0 < (float)H ? (int)cy0 : H) : 0;
                y1p = cy1 < (float)(H - 1) ? (cy1 >= -1.0f ? (int)cy1 : -1) : H - 1;
            }
            if (x0p <= x1p && y0p <= y1p) {
                const unsigned* S = sat + sat_off;
                const size_t w1 = (size_t)W + 1;
                const unsigned cnt = S[(size_t)(y1p + 1) * w1 + (x1p + 1)] - S[(size_t)y0p * w1 + (x1p + 1)] -
                                     S[(size_t)(y1p + 1) * w1 + x0p] + S[(size_t)y0p * w1 + x0p];
                if (cnt) tag |= 1u << v;
            }
        }
        __syncthreads();
        sat_off += (size_t)(H + 1) * (W + 1);
    }
    if (live) tags[((long long)k * ny + j) * nx + i] = tag;
}

cudaError_t launch_visual_hull(const CamDev* cams, int ncam, int W, int H, int nx, int ny, int nz,
                               const float* targets, float thresh, unsigned* sat, unsigned* tags, cudaStream_t s)
{
    HullCams hc;
    for (int v = 0; v < ncam; ++v) hc.c[v] = cams[v];
    const int rows = ncam * (H + 1), tiles = (W + 1 + 31) / 32;
    sat_rows_kernel<<<(unsigned)((rows + 7) / 8), 256, 0, s>>>(targets, ncam, W, H, thresh, sat);
    sat_cols_kernel<<<(unsigned)(ncam * tiles), dim3(32, kSatChunks), 0, s>>>(ncam, W, H, sat);
    const long long node_tiles = (long long)((nx + kHullTX - 1) / kHullTX) * ((ny + kHullTY - 1) / kHullTY) *
                                 ((nz + kHullTZ - 1) / kHullTZ);
    hull_kernel<<<(unsigned)node_tiles, kHullTX * kHullTY * kHullTZ, 0, s>>>(hc, ncam, nx, ny, nz, sat, tags);
    return cudaGetLastError();
}

// Records outside the hull (tag != full) are set to 0: no emission, no
// extinction (vol null: nothing is cleared).  With `flags`, also marks the
// bricks of kBrick^3 cells that hold a key point inside the hull (the flags are
// cleared beforehand).
template <int DT>
__global__ void __launch_bounds__(256) hull_clear_kernel(void* vol, int nx, int ny, int nz,
                                                         const unsigned* __restrict__ tags, unsigned full,
                                                         unsigned char* flags, int nbx, int nby, int nbz)
{
    const long long nodes = (long long)nx * ny * nz;
    // box of the bricks this thread flags (merged into the table's box below)
    unsigned lo[3] = {UINT_MAX, UINT_MAX, UINT_MAX}, hi[3] = {0u, 0u, 0u};
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < nodes;
         i += (long long)gridDim.x * blockDim.x) {
        if (__ldg(tags + i) != full) {
            if (vol) store_rgb<DT>(vol, i, make_float4(0.0f, 0.0f, 0.0f, 0.0f));
        } else if (flags) {
            const unsigned row = (unsigned)i / (unsigned)nx, zu = row / (unsigned)ny;
            const int x = (int)((unsigned)i - row * (unsigned)nx), y = (int)(row - zu * (unsigned)ny), z = (int)zu;
            mark_bricks(flags, x, y, z, nbx, nby, nbz);
            const int c[3] = {x, y, z}, nb[3] = {nbx, nby, nbz};
#pragma unroll
            for (int a = 0; a < 3; ++a) {
                constexpr int S = kBrickShift, M = kBrick - 1;
                const int b0 = (c[a] > 0 && (c[a] & M) == 0) ? (c[a] >> S) - 1 : (c[a] >> S);
                lo[a] = min(lo[a], (unsigned)b0);
                hi[a] = max(hi[a], (unsigned)min(c[a] >> S, nb[a] - 1) + 1u);
            }
        }
    }
    if (flags) merge_box(flags, nbx, nby, nbz, lo, hi);
}

cudaError_t launch_hull_clear(void* vol, int dt, int nx, int ny, int nz, const unsigned* tags, unsigned full,
                              unsigned char* flags, cudaStream_t s)
{
    const int nbx = bricks_along(nx), nby = bricks_along(ny), nbz = bricks_along(nz);
    if (flags) {
        cudaError_t e = cudaMemsetAsync(flags, 0, brick_table_bytes(nx, ny, nz), s);
        if (e != cudaSuccess) return e;
    }
    const long long nodes = (long long)nx * ny * nz;
    const int g = grid_for(nodes, 256);
#define FR_CLEAR(D) hull_clear_kernel<D><<<g, 256, 0, s>>>(vol, nx, ny, nz, tags, full, flags, nbx, nby, nbz)
    if (dt == DT_F32) FR_CLEAR(DT_F32);
    else if (dt == DT_BF16) FR_CLEAR(DT_BF16);
    else FR_CLEAR(DT_F16);
#undef FR_CLEAR
    return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// Error measure and fills
// ---------------------------------------------------------------------------

// Temperature from the green channel (Sec. 3.3.3): per node, the inverse of
// the table's piecewise-linear green column (bisection over its m entries,
// strictly increasing), clamped to [t_min, t_max]; the extinction is copied.
template <int DR, int DT>
__global__ void __launch_bounds__(256) green_to_temp_kernel(const void* rgb, void* temp, long long nodes,
                                                            const float4* __restrict__ lut, int m, float t_min,
                                                            float t_max)
{
    const float g_lo = __ldg(&lut[0].y), g_hi = __ldg(&lut[m - 1].y);
    const float dt = (t_max - t_min) / (float)(m - 1);
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < nodes;
         i += (long long)gridDim.x * blockDim.x) {
        const float4 r = load_rgb<DR>(rgb, i);
        const float g = r.y;
        float t;
        if (!(g > g_lo)) {
            t = t_min;
        } else if (!(g < g_hi)) {
            t = t_max;
        } else {
            int lo = 0, hi = m - 1;   // lut[lo].y < g < lut[hi].y
            while (hi - lo > 1) {
                const int mid = lo + ((hi - lo) >> 1);
                if (__ldg(&lut[mid].y) <= g) lo = mid;
                else hi = mid;
            }
            const float a = __ldg(&lut[lo].y), b = __ldg(&lut[hi].y);
            t = t_min + ((float)lo + (g - a) / (b - a)) * dt;
        }
        store_ts<DT>(temp, i, make_float2(t, r.w));
    }
}

cudaError_t launch_green_to_temp(const void* rgb, int dt_rgb, void* temp, int dt_temp, long long nodes,
                                 const float* lut, int m, float t_min, float t_max, cudaStream_t s)
{
    const int g = grid_for(nodes, 256);
    const float4* l4 = reinterpret_cast<const float4*>(lut);
#define FR_G2T(DR, DT) green_to_temp_kernel<DR, DT><<<g, 256, 0, s>>>(rgb, temp, nodes, l4, m, t_min, t_max)
#define FR_G2T_T(DR)                                \
    if (dt_temp == DT_F32) FR_G2T(DR, DT_F32);      \
    else if (dt_temp == DT_BF16) FR_G2T(DR, DT_BF16); \
    else FR_G2T(DR, DT_F16)
    if (dt_rgb == DT_F32) { FR_G2T_T(DT_F32); }
    else if (dt_rgb == DT_BF16) { FR_G2T_T(DT_BF16); }
    else { FR_G2T_T(DT_F16); }
#undef FR_G2T_T
#undef FR_G2T
    return cudaGetLastError();
}

// Volume data error (Sec. 5.1): squared emission differences of two volumes
// summed per CTA over the key points inside the hull (tags == full; all when
// tags is null), then summed over the CTAs in a fixed order.
struct ErrPartial {
    float s[3];
    unsigned n;
};

template <int DA, int DB>
__global__ void __launch_bounds__(256) volume_err_kernel(const void* a, const void* b, long long nodes,
                                                         const unsigned* __restrict__ tags, unsigned full,
                                                         ErrPartial* partials)
{
    __shared__ float red[3][8];
    __shared__ unsigned redn[8];
    float s0 = 0.0f, s1 = 0.0f, s2 = 0.0f;
    unsigned n = 0;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < nodes;
         i += (long long)gridDim.x * blockDim.x) {
        if (tags && __ldg(tags + i) != full) continue;
        const float4 va = load_rgb<DA>(a, i), vb = load_rgb<DB>(b, i);
        const float d0 = va.x - vb.x, d1 = va.y - vb.y, d2 = va.z - vb.z;
        s0 = fmaf(d0, d0, s0); s1 = fmaf(d1, d1, s1); s2 = fmaf(d2, d2, s2);
        ++n;
    }
    s0 = warp_sum(s0); s1 = warp_sum(s1); s2 = warp_sum(s2);
    n = __reduce_add_sync(0xffffffffu, n);
    const int w = threadIdx.x >> 5;
    if ((threadIdx.x & 31) == 0) { red[0][w] = s0; red[1][w] = s1; red[2][w] = s2; redn[w] = n; }
    __syncthreads();
    if (threadIdx.x == 0) {
        ErrPartial p{{0.0f, 0.0f, 0.0f}, 0u};
        for (int i = 0; i < (int)(blockDim.x >> 5); ++i) {
            p.s[0] += red[0][i]; p.s[1] += red[1][i]; p.s[2] += red[2][i]; p.n += redn[i];
        }
        partials[blockIdx.x] = p;
    }
}

// out: rmse3 (3 floats) then the count (unsigned long long at byte 16).
__global__ void __launch_bounds__(1024) volume_err_finish(const ErrPartial* partials, int np, float* out)
{
    __shared__ float red[3][32];
    __shared__ unsigned long long redn[32];
    float s0 = 0.0f, s1 = 0.0f, s2 = 0.0f;
    unsigned long long n = 0;
    for (int i = threadIdx.x; i < np; i += blockDim.x) {
        const ErrPartial p = partials[i];
        s0 += p.s[0]; s1 += p.s[1]; s2 += p.s[2]; n += p.n;
    }
    s0 = warp_sum(s0); s1 = warp_sum(s1); s2 = warp_sum(s2);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) n += __shfl_xor_sync(0xffffffffu, n, o);
    const int w = threadIdx.x >> 5;
    if ((threadIdx.x & 31) == 0) { red[0][w] = s0; red[1][w] = s1; red[2][w] = s2; redn[w] = n; }
    __syncthreads();
    if (threadIdx.x == 0) {
        float t[3] = {0.0f, 0.0f, 0.0f};
        unsigned long long tn = 0;
        for (int i = 0; i < (int)(blockDim.x >> 5); ++i) {
            t[0] += red[0][i]; t[1] += red[1][i]; t[2] += red[2][i]; tn += redn[i];
        }
        for (int c = 0; c < 3; ++c) out[c] = tn ? sqrtf(t[c] / (float)tn) : 0.0f;
        *reinterpret_cast<unsigned long long*>(out + 4) = tn;
    }
}

int volume_err_blocks(long long nodes) { return grid_for(nodes, 256); }

cudaError_t launch_volume_err(const void* a, int dta, const void* b, int dtb, long long nodes, const unsigned* tags,
                              unsigned full, void* partials, float* out, cudaStream_t s)
{
    const int g = grid_for(nodes, 256);
    ErrPartial* pp = static_cast<ErrPartial*>(partials);
#define FR_ERR(DA, DB) volume_err_kernel<DA, DB><<<g, 256, 0, s>>>(a, b, nodes, tags, full, pp)
#define FR_ERR_B(DA)                              \
    if (dtb == DT_F32) FR_ERR(DA, DT_F32);        \
    else if (dtb == DT_BF16) FR_ERR(DA, DT_BF16); \
    else FR_ERR(DA, DT_F16)
    if (dta == DT_F32) { FR_ERR_B(DT_F32); }
    else if (dta == DT_BF16) { FR_ERR_B(DT_BF16); }
    else { FR_ERR_B(DT_F16); }
#undef FR_ERR_B
#undef FR_ERR
    volume_err_finish<<<1, 1024, 0, s>>>(pp, g, out);
    return cudaGetLastError();
}

// End of one iteration of a device-counted loop (one thread): the image error
// of iteration it = *iter from its squared-error sums (255 sqrt(sum / count)), the
// stop criterion |E_it - E_it-1| < stop_delta in every channel (or the last
// allowed iteration) ending the conditional loop, the counter advanced and the
// flame-ray count cleared for the next forward march.
__global__ void converge_kernel(const float* __restrict__ sq4, float* hist3, int* iter, unsigned* flame_count,
                                int n_counts, int max_iters, float stop_delta, cudaGraphConditionalHandle handle)
{
    if (threadIdx.x != 0 || blockIdx.x != 0) return;
    const int it = *iter;
    if (it < 0 || it >= max_iters) {   // never expected: end the loop rather than write out of range
        cudaGraphSetConditional(handle, 0u);
        return;
    }
    const float cnt = sq4[3];
    float r[3];
#pragma unroll
    for (int c = 0; c < 3; ++c) r[c] = cnt > 0.0f ? 255.0f * sqrtf(sq4[c] / cnt) : 0.0f;
    bool stop = it + 1 >= max_iters;
    if (it >= 1) {
        bool small = true;
#pragma unroll
        for (int c = 0; c < 3; ++c) small = small && fabsf(r[c] - hist3[3 * (it - 1) + c]) < stop_delta;
        stop = stop || small;
    }
#pragma unroll
    for (int c = 0; c < 3; ++c) hist3[3 * it + c] = r[c];
    *iter = it + 1;
    if (flame_count)
        for (int i = 0; i < n_counts; ++i) flame_count[i] = 0u;
    if (stop) cudaGraphSetConditional(handle, 0u);
}

cudaError_t launch_converge(const float* sq4, float* hist3, int* iter, unsigned* flame_count, int n_counts,
                            int max_iters, float stop_delta, cudaGraphConditionalHandle handle, cudaStream_t s)
{
    converge_kernel<<<1, 32, 0, s>>>(sq4, hist3, iter, flame_count, n_counts, max_iters, stop_delta, handle);
    return cudaGetLastError();
}

__global__ void fill_kernel(float* p, long long n, float v)
{
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
        p[i] = v;
}

cudaError_t launch_fill(float* p, long long n, float v, cudaStream_t s)
{
    fill_kernel<<<grid_for(n, 256), 256, 0, s>>>(p, n, v);
    return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// Storage conversion of a volume's records (fr_volume_upload / download):
// float32 values to and from the 16-bit storage types, rounding to nearest
// even.  Streaming: four values (16 bytes of float32) per thread and step;
// a count that is not a multiple of 4 leaves two values for the last thread.
// ---------------------------------------------------------------------------

template <int DT>
__device__ __forceinline__ uint32_t pack2(float a, float b)
{
    if constexpr (DT == DT_BF16) {
        const __nv_bfloat162 h = __floats2bfloat162_rn(a, b);
        return *reinterpret_cast<const uint32_t*>(&h);
    } else {
        const __half2 h = __floats2half2_rn(a, b);
        return *reinterpret_cast<const uint32_t*>(&h);
    }
}

template <int DT>
__device__ __forceinline__ float2 unpack2(uint32_t u)
{
    if constexpr (DT == DT_BF16) return make_float2(bf16_lo(u), bf16_hi(u));
    else return f16x2(u);
}

template <int DT>
__global__ void __launch_bounds__(256) to_storage_kernel(const float* __restrict__ src, void* dst, long long n)
{
    const long long quads = n >> 2;
    const float4* s4 = reinterpret_cast<const float4*>(src);
    uint2* d4 = reinterpret_cast<uint2*>(dst);
    const long long stride = (long long)gridDim.x * blockDim.x;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < quads; i += stride) {
        const float4 v = __ldg(s4 + i);
        d4[i] = make_uint2(pack2<DT>(v.x, v.y), pack2<DT>(v.z, v.w));
    }
    if ((n & 3) && blockIdx.x == 0 && threadIdx.x == 0) {
        const long long at = quads * 4;
        reinterpret_cast<uint32_t*>(dst)[at >> 1] = pack2<DT>(src[at], src[at + 1]);
    }
}

template <int DT>
__global__ void __launch_bounds__(256) from_storage_kernel(const void* src, float* __restrict__ dst, long long n)
{
    const long long quads = n >> 2;
    const uint2* s4 = reinterpret_cast<const uint2*>(src);
    float4* d4 = reinterpret_cast<float4*>(dst);
    const long long stride = (long long)gridDim.x * blockDim.x;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < quads; i += stride) {
        const uint2 u = __ldg(s4 + i);
        const float2 a = unpack2<DT>(u.x), b = unpack2<DT>(u.y);
        d4[i] = make_float4(a.x, a.y, b.x, b.y);
    }
    if ((n & 3) && blockIdx.x == 0 && threadIdx.x == 0) {
        const long long at = quads * 4;
        const float2 a = unpack2<DT>(reinterpret_cast<const uint32_t*>(src)[at >> 1]);
        dst[at] = a.x;
        dst[at + 1] = a.y;
    }
}

cudaError_t launch_to_storage(const float* src, void* dst, int dt, long long n, cudaStream_t s)
{
    const int g = grid_for((n + 3) / 4, 256);
    if (dt == DT_BF16) to_storage_kernel<DT_BF16><<<g, 256, 0, s>>>(src, dst, n);
    else if (dt == DT_F16) to_storage_kernel<DT_F16><<<g, 256, 0, s>>>(src, dst, n);
    else return cudaErrorInvalidValue;
    return cudaGetLastError();
}

cudaError_t launch_from_storage(const void* src, float* dst, int dt, long long n, cudaStream_t s)
{
    const int g = grid_for((n + 3) / 4, 256);
    if (dt == DT_BF16) from_storage_kernel<DT_BF16><<<g, 256, 0, s>>>(src, dst, n);
    else if (dt == DT_F16) from_storage_kernel<DT_F16><<<g, 256, 0, s>>>(src, dst, n);
    else return cudaErrorInvalidValue;
    return cudaGetLastError();
}

cudaError_t check_word_volume(unsigned* word, bool reset)
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
