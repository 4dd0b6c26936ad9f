// fr_internal.h -- launchers shared by the library's translation units.
#pragma once

#include <cuda_runtime.h>

#include "fr_device.cuh"

namespace frk {

constexpr int kMaxViews = 32;

// Kernel argument block of single-problem launches: the problem and its
// cameras travel by value in the kernel's parameter space (no device copy).
struct SingleArgs {
    ProbDev p;
    CamDev cams[kMaxViews];
};

inline int tiles_of(int W, int H, int ncam)
{
    return ((W + kTileW - 1) / kTileW) * ((H + kTileH - 1) / kTileH) * ncam;
}

// march.cu
cudaError_t launch_fwd(const SingleArgs& a, int dt, int kind, int ntiles, cudaStream_t s);
// The forward march's tiles longest first (for a.p.tile_order): key and order
// hold ntiles words each; box (brick-table layout, nullable) bounds the
// samples counted per ray.
#ifndef FR_MARCH_ORDER
#define FR_MARCH_ORDER 1
#endif
cudaError_t launch_tile_order(const SingleArgs& a, int ntiles, const unsigned* box, unsigned* key,
                              unsigned* order, cudaStream_t s);
#ifndef FR_FUSED
#define FR_FUSED 0
#endif
#if FR_FUSED
// forward march and paper-rule adjustment of each tile in one kernel (RGB
// x-pair records with brick skipping; a.p carries the forward's and the
// adjustment's fields, no residual image and no flame list; the comparison
// variant of march.cu's fwd_single + adj_list)
cudaError_t launch_fused(const SingleArgs& a, int dt, int ntiles, cudaStream_t s);
#endif
// Loads the kernels the allocation-free render launches (the forward march
// gathering records one by one, every storage type, kind and opacity mode,
// and the one-CTA error reduction) on the current device, so that their first
// launch needs no module loading.
cudaError_t preload_noalloc_kernels();
cudaError_t launch_fwd_batch(const ProbDev* probs, const int* tile_start, int nprob, int total_tiles,
                             int dt, int kind, bool tau, bool pairs, cudaStream_t s, bool skip = false);
// x-pair records of every problem's volume (vol_rw -> pairs), RGB records
cudaError_t launch_pair_pack_batch(const ProbDev* probs, int nprob, int dt, cudaStream_t s);
cudaError_t launch_adjust(const SingleArgs& a, int dt, int ntiles, cudaStream_t s);
// Parts a batched problem's flame rays are adjusted in (march.cu: 1 unless
// built with -DFR_BATCH_PARTS=FR_ADJ_SPLIT)
#ifndef FR_BATCH_PARTS
#define FR_BATCH_PARTS 1
#endif
// parts > 1: every problem's flame list holds that many entries per ray
// (launch_flame_list with the same parts) and ProbDev::tpart is set
cudaError_t launch_adjust_list_batch(const ProbDev* probs, const int* tile_start, int nprob, int total_tiles,
                                     int dt, bool tau, int iteration, cudaStream_t s, bool skip = false,
                                     int parts = 1);
cudaError_t launch_finalize_batch(const ProbDev* probs, int nprob, int iteration, cudaStream_t s);
cudaError_t launch_apply_batch(const ProbDev* probs, int nprob, int dt, int clamp_nonneg, cudaStream_t s);
// batched brick tables (P.occ: flags cleared, then their box); the batched
// update clears the records outside each problem's hull (P.hull)
cudaError_t launch_brick_reset_batch(const ProbDev* probs, int nprob, cudaStream_t s);
cudaError_t launch_brick_box_batch(const ProbDev* probs, int nprob, cudaStream_t s);
cudaError_t launch_rmse_batch(const ProbDev* probs, int nprob, int iters, float* rmse_all, cudaStream_t s);
cudaError_t launch_backward(const SingleArgs& a, int dt, int kind, int ntiles, cudaStream_t s);
cudaError_t launch_backward_batch(const ProbDev* probs, const int* tile_start, int nprob, int total_tiles,
                                  int dt, int kind, bool tau, cudaStream_t s);
cudaError_t launch_count(const SingleArgs& a, int ntiles, cudaStream_t s);
// scratch (nullable): kFinScratchBytes of device memory, kFinParts float4 and
// then a counter word that is 0 before the first launch (every launch leaves
// it 0); with it the sum runs over kFinParts CTAs, without it in one.  rmse3
// (nullable, with scratch only): the error measure of the final sums (Sec.
// 5.1), 255 sqrt(sum / count) per channel, 0 without counted pixels.
constexpr int kFinParts = 32;
constexpr size_t kFinScratchBytes = kFinParts * 16 + 16;
cudaError_t launch_finalize(const float* partials, int ntiles, float* out4, cudaStream_t s, int accumulate = 0,
                            void* scratch = nullptr, float* rmse3 = nullptr);
// flame-ray list of a problem with prepared targets: buf needs
// flame_list_buf_entries(ntiles) entries, the total lands at
// buf[flame_list_total_at(ntiles)]; list needs parts entries per pixel at
// most (parts > 1: one entry per part of each ray, the part in the top two
// bits, each tile's run one padded block per part)
inline size_t flame_list_buf_entries(int ntiles) { return (size_t)ntiles * (kTileThreads / 32 + 1) + 1; }
inline size_t flame_list_total_at(int ntiles) { return (size_t)ntiles * (kTileThreads / 32 + 1); }
cudaError_t launch_flame_list(const SingleArgs& a, int ntiles, unsigned* buf, unsigned* list, cudaStream_t s,
                              int parts = 1);
#ifdef FR_ADJ_GATHER_PROBE
// lower-bound measurement of a gather adjustment (march.cu): list and sink
// hold one entry per node, count one word
cudaError_t launch_gather_probe(const SingleArgs& a, const unsigned* tags, unsigned full, long long nodes,
                                unsigned* list, unsigned* count, float* sink, cudaStream_t s);
#endif
// tm (nullable): the list holds both halves of every flame ray (ProbDev::flist_tm)
cudaError_t launch_adjust_list(const SingleArgs& a, int dt, int ntiles, const unsigned* list,
                               const unsigned* count, cudaStream_t s, const float* tm = nullptr);

// tables.cu: the paper-rule loop over a fixed extinction field as a forward
// table (per ray: key point, A) and an adjustment table (per key point of the
// hull: flame ray, W), built by two marches over every ray.
// 3D Morton codes: bit i of a coordinate goes to bit 3 i (+0 x, +1 y, +2 z)
// of the code; coordinates below 2^21.
__host__ __device__ inline unsigned long long morton_spread(unsigned v)
{
    unsigned long long x = v & 0x1fffffull;
    x = (x | x << 32) & 0x1f00000000ffffull;
    x = (x | x << 16) & 0x1f0000ff0000ffull;
    x = (x | x << 8) & 0x100f00f00f00f00full;
    x = (x | x << 4) & 0x10c30c30c30c30c3ull;
    x = (x | x << 2) & 0x1249249249249249ull;
    return x;
}
__host__ __device__ inline unsigned morton_compact(unsigned long long x)
{
    x &= 0x1249249249249249ull;
    x = (x ^ (x >> 2)) & 0x10c30c30c30c30c3ull;
    x = (x ^ (x >> 4)) & 0x100f00f00f00f00full;
    x = (x ^ (x >> 8)) & 0x1f0000ff0000ffull;
    x = (x ^ (x >> 16)) & 0x1f00000000ffffull;
    x = (x ^ (x >> 32)) & 0x1fffffull;
    return (unsigned)x;
}
// The order the tables list key points in: item i of [0, count()) names
// node(i), or -1 for an item outside the grid.  mbits > 0: Morton order over
// a cube of 2^mbits nodes per edge; 0: node order.
struct KeyOrder {
    int nx = 0, ny = 0, nz = 0, mbits = 0;
    __host__ __device__ long long count() const
    {
        return mbits ? 1LL << (3 * mbits) : (long long)nx * ny * nz;
    }
    __device__ long long node(long long i) const
    {
        if (!mbits) return i;
        const unsigned long long c = (unsigned long long)i;
        const unsigned x = morton_compact(c), y = morton_compact(c >> 1), z = morton_compact(c >> 2);
        if (x >= (unsigned)nx || y >= (unsigned)ny || z >= (unsigned)nz) return -1;
        return ((long long)z * ny + y) * nx + x;
    }
};

struct TabBuild {
    const unsigned* tags;   // visual hull tags; key points whose tag is `full` are inside
    unsigned full;
    unsigned* wrows;        // per warp of the tiles: rows of its forward entries
    unsigned* woff;         // per warp: first row
    unsigned* tfl;          // per tile: flame rays
    unsigned* tfoff;        // per tile: number of its first flame ray
    unsigned* ncnt;         // per node: adjustment entries (count pass), then the next free one (fill pass)
    unsigned* hnode;        // the hull's key points in the listing order
    unsigned* hid;          // per node inside the hull: its place in that list
    const unsigned* torder; // the fill's tiles in launch order (nullable: tile order)
    KeyOrder order;
    long long nodes;
    uint2* efwd;            // forward entries {place in the hull's list, A}
    uint2* eadj;            // adjustment entries {flame ray, W}
    unsigned long long nadj;
    unsigned nhull;         // key points inside the hull (fill pass)
};
struct TabIter {
    const unsigned* wrows;
    const unsigned* woff;
    const unsigned* tfoff;
    const uint2* efwd;
    const uint2* eadj;
    const unsigned* hnode;
    const unsigned* hend;   // per key point of the hull: end of its entries
    void* hs;               // per key point of the hull: its source record (the forward's gather)
    float4* dl;             // per flame ray: its residual {r, g, b, 0}
    const unsigned* torder; // the forward's tiles in launch order (nullable: tile order)
    unsigned nhull, nflame, nadj;
};
// a.p: the problem with targets, cameras and the hull's brick table
// (adj_occ, adj_box); a.p.vol the records whose extinction fixes T.
cudaError_t launch_tab_count(const SingleArgs& a, const TabBuild& b, int dt, int ntiles, cudaStream_t s);
// exclusive scans of the counts: totals[0] rows, [1] flame rays, [2]
// adjustment entries, [3] key points inside the hull (bsum:
// tab_scan_blocks(max(warps, b.order.count())) words); then b.hid of the
// listed key points
cudaError_t launch_tab_scans(const TabBuild& b, int ntiles, unsigned long long* bsum, unsigned long long* totals,
                             cudaStream_t s);
size_t tab_scan_blocks(long long n);
cudaError_t launch_tab_fill(const SingleArgs& a, const TabBuild& b, int dt, int ntiles, cudaStream_t s);
cudaError_t launch_tab_hend(const unsigned* hnode, const unsigned* cursor, unsigned nh, unsigned* hend,
                            cudaStream_t s);
// each key point's adjustment entries in increasing flame-ray order (FR_TAB_SORT builds)
cudaError_t launch_tab_sort(uint2* eadj, const unsigned* hend, unsigned nh, cudaStream_t s);
// it.hs[h] = records[it.hnode[h]] (records: the volume's storage type)
cudaError_t launch_tab_stage(const void* records, int dt, const TabIter& it, cudaStream_t s);
// a.p.vol: the source records; targets, bbox and partials as for the forward
// march (rendered and residual images when set)
cudaError_t launch_tab_forward(const SingleArgs& a, const TabIter& it, int dt, int ntiles, cudaStream_t s);
// The tables' iterations sum the forward's errors inside the adjustment's
// launch (FR_TAB_FIN_FUSED = 0: a launch of their own between the two).
#ifndef FR_TAB_FIN_FUSED
#define FR_TAB_FIN_FUSED 1
#endif
// The error sums of a forward pass run by kFinParts extra CTAs of another
// launch (finalize_parts_body): the tiles' partials, the sums written to out4
// (not accumulated), the error measure to rmse3 (nullable); scratch as for
// launch_finalize (kFinScratchBytes, its counter word 0).
struct FinArgs {
    const float* partials;
    int ntiles;
    float* out4;
    void* scratch;
    float* rmse3;
};
// the adjustment added to the hull's key points of vol (RGB records); fin
// (nullable): the forward's error sums in the same launch, the update needing
// only the residuals
cudaError_t launch_tab_adjust(void* vol, int dt, long long nodes, const TabIter& it, int clamp_nonneg,
                              cudaStream_t s, const FinArgs* fin = nullptr);
cudaError_t check_word_tables(unsigned* word, bool reset);
// Several problems' tables per launch (the server): tile_start / blk_start
// ascending with the total last (blocks of the adjustment: tab_adjust_blocks
// of a problem's key points); the batched adjustment updates each P.vol_rw
// and writes the updated records to its.hs, the next iteration's staged
// source (problems without in-scattering).
unsigned tab_adjust_blocks(unsigned nh);
cudaError_t launch_tab_forward_batch(const ProbDev* probs, const TabIter* its, const int* tile_start, int nprob,
                                     int total_tiles, int dt, cudaStream_t s);
cudaError_t launch_tab_adjust_batch(const ProbDev* probs, const TabIter* its, const int* blk_start, int nprob,
                                    int total_blocks, int dt, int clamp_nonneg, cudaStream_t s);
// host: the forward's tiles in launch order from the warps' rows (the tile
// with the most rows in one warp first; FR_TAB_LPT = 0: tile order)
void tab_tile_order(const unsigned* wrows, int ntiles, unsigned* order);

// volume.cu
cudaError_t launch_apply(void* vol, int dt, int kind, long long nodes, float* dV, float scale,
                         int with_sigma, int clamp_nonneg, int zero_dV, cudaStream_t s,
                         const unsigned* hull = nullptr, unsigned hull_full = 0);
// The box of a brick table's flagged bricks (brick-table layout, on the
// device; see brick_box) taken as the range of nodes that are corners of
// their cells.  box == nullptr: the whole grid.
struct NodeBox {
    const unsigned* box = nullptr;
    int nbx = 0, nby = 0, nbz = 0;
};
// x-pair records and brick marks written by the last in-scattering sweep
// (the pair pack folded into it): pair i = {source i, source of its +x
// neighbour}, the second half repeating the first on the box's last x; occ
// (cleared beforehand) flags the bricks of every non-zero source record.
struct PackOut {
    void* pairs = nullptr;
    unsigned char* occ = nullptr;
};
// Whether launch_scatter_source honours a NodeBox (and a PackOut) for this grid.
bool sweeps_take_box(int nx, int ny, int nz);
// launch_apply over the nodes of `box` only (the whole grid without one): the
// caller guarantees that every record and every update outside it is zero.
cudaError_t launch_apply_box(void* vol, int dt, int kind, int nx, int ny, int nz, float* dV, float scale,
                             int with_sigma, int clamp_nonneg, int zero_dV, cudaStream_t s, const unsigned* hull,
                             unsigned hull_full, NodeBox box);
// skip_empty: chunks of a grid line whose records are all zero skip their
// walks; J is then left undefined at their nodes (their source is 0 anyway),
// so only the reconstruction loop, which reads the source alone, asks for it.
// box: every record outside it is zero, and J and the source are computed at
// its nodes only (left undefined elsewhere; grids whose lines run the
// register-held chunks, the others in full).
// pk (with a box the sweeps honour): the pairs and brick marks of the source
// records at the box's nodes, as launch_pair_pack with that box would write
// them for the forward march.
cudaError_t launch_scatter_source(const void* emission, int dt_in, const float* albedo, float* J,
                                  void* out, int dt_out, int nx, int ny, int nz, cudaStream_t s,
                                  bool skip_empty = false, NodeBox box = NodeBox{}, PackOut pk = PackOut{});
cudaError_t launch_planck_lut(float t_min, float t_max, int m, float* lut, cudaStream_t s);
cudaError_t launch_prepare_targets(float* targets, int ncam, int H, int W, float thresh, int* bbox,
                                   cudaStream_t s);
// temperature records {T, sigma} from the green channel of RGB records
cudaError_t launch_green_to_temp(const void* rgb, int dt_rgb, void* temp, int dt_temp, long long nodes,
                                 const float* lut, int m, float t_min, float t_max, cudaStream_t s);
// volume data error of two RGB volumes' emission inside the hull: partials
// (volume_err_blocks(nodes) x 16 bytes), out = rmse3, then the count as a
// 64-bit integer at float offset 4
int volume_err_blocks(long long nodes);
cudaError_t launch_volume_err(const void* a, int dta, const void* b, int dtb, long long nodes, const unsigned* tags,
                              unsigned full, void* partials, float* out, cudaStream_t s);
// bounds-check words of the checked build (0 otherwise), per translation unit
cudaError_t check_word_march(unsigned* word, bool reset);
cudaError_t check_word_volume(unsigned* word, bool reset);
// end of an iteration of a loop counted on the device (conditional graph body);
// clears flame_count[0 .. n_counts)
cudaError_t launch_converge(const float* sq4, float* hist3, int* iter, unsigned* flame_count, int n_counts,
                            int max_iters, float stop_delta, cudaGraphConditionalHandle handle, cudaStream_t s);
// In-scattering with a Henyey-Greenstein phase function: the six directional
// radiances per node (L6, nodes x 6 float4, d = 2 axis + (0: +axis, 1: -axis)),
// and the source towards one view, S = q + albedo sigma sum_d w_d L_d.
cudaError_t launch_scatter_L6(const void* emission, int dt, float* L6, int nx, int ny, int nz, cudaStream_t s,
                              bool skip_empty = false);
struct HgWeights {
    float w[6];
};
cudaError_t launch_source_hg(const void* emission, int dt, const float* albedo, const float* L6, HgWeights w,
                             void* out, long long nodes, cudaStream_t s);
cudaError_t launch_fill(float* p, long long n, float v, cudaStream_t s);
// n float32 values (even; 8-byte aligned source, 16-byte aligned for the
// vector path) to and from the 16-bit storage type dt, rounding to nearest even
cudaError_t launch_to_storage(const float* src, void* dst, int dt, long long n, cudaStream_t s);
cudaError_t launch_from_storage(const void* src, float* dst, int dt, long long n, cudaStream_t s);
// visual hull: sat needs ncam (H+1)(W+1) uint32, tags one uint32 per node
cudaError_t launch_visual_hull(const CamDev* cams, int ncam, int W, int H, int nx, int ny, int nz,
                               const float* targets, float thresh, unsigned* sat, unsigned* tags, cudaStream_t s);
// Records outside the hull (tag != full) set to 0 (vol null: none); with
// flags, the brick table of the key points inside the hull
cudaError_t launch_hull_clear(void* vol, int dt, int nx, int ny, int nz, const unsigned* tags, unsigned full,
                              unsigned char* flags, cudaStream_t s);
// Brick tables: one flag per brick of kBrick^3 cells (x fastest), then, at the
// next 16-byte boundary, the box of the flagged bricks as six unsigned
// values {nbx - lo_x, nby - lo_y, nbz - lo_z, hi_x + 1, hi_y + 1, hi_z + 1}
// (all 0 when no brick is flagged).
__host__ __device__ inline int bricks_along(int n) { return (n - 2) / kBrick + 1; }
__host__ __device__ inline size_t brick_count(int nx, int ny, int nz)
{
    return (size_t)bricks_along(nx) * bricks_along(ny) * bricks_along(nz);
}
__host__ __device__ inline size_t brick_box_offset(int nx, int ny, int nz)
{
    return (brick_count(nx, ny, nz) + 15) & ~(size_t)15;
}
__host__ __device__ inline size_t brick_table_bytes(int nx, int ny, int nz) { return brick_box_offset(nx, ny, nz) + 32; }
__host__ __device__ inline unsigned* brick_box(unsigned char* table, int nbx, int nby, int nbz)
{
    return reinterpret_cast<unsigned*>(table + (((size_t)nbx * nby * nbz + 15) & ~(size_t)15));
}
// x-pair records of a volume (2 records per node) for the forward march, and
// (occ non-null, RGB records) the brick table of its non-zero records.  keep
// (nullable, brick-table layout): only nodes of flagged bricks are packed and
// their box is the one the forward clips to, so occ's own box is not computed
// (for the visual hull's table, whose flagged-off bricks hold zero records).
// box (with keep): the records are known inside it only (launch_scatter_source
// with that box) and are zero outside; nodes outside are not packed.
cudaError_t launch_pair_pack(const void* src, void* dst, int dt, int kind, int nx, int ny, int nz,
                             unsigned char* occ, cudaStream_t s, const unsigned char* keep = nullptr,
                             NodeBox box = NodeBox{});

}  // namespace frk
