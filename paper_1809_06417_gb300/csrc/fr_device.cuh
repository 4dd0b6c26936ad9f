// fr_device.cuh -- device-side building blocks of the flame reconstruction
// kernels: camera rays, box clipping, node-record loads for each storage type,
// trilinear sampling, the colour-temperature table and the G(s) stream.
//
// Conventions (identical to the C ABI, include/flamerec.h): key points are
// grid nodes (Sec. 3.3 definitions); all ray arithmetic is in voxel units;
// a ray is cut into segments of length `step` from its box entry point and
// each segment is sampled at its midpoint.
#pragma once

#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <cuda_runtime.h>
#include <stdint.h>

// Parts the adjustment splits each flame ray into (the samples before and
// after the ray's middle sample, the second part starting from the
// transmittance the forward march reached there): twice as many, shorter work
// items, so the kernel's last wave, in which SMs run out of rays, is shorter
// (2 parts measured 6% faster than whole rays; 3 parts 11% and 4 parts 23%
// slower than 2).  1 lists whole rays.
#ifndef FR_ADJ_SPLIT
#define FR_ADJ_SPLIT 2
#endif
static_assert(FR_ADJ_SPLIT >= 1 && FR_ADJ_SPLIT <= 4, "FR_ADJ_SPLIT: 1 to 4 parts (two bits of a list entry)");

namespace frk {

enum { DT_F32 = 0, DT_BF16 = 1, DT_F16 = 2 };
enum { KIND_RGB = 0, KIND_TEMP = 1 };

// Pixel tile of one CTA: 16 x 8 rays, one per thread; each warp marches an
// 8 x 4 sub-tile so that its rays stay close together inside the volume.
constexpr int kTileW = 16;
#ifndef FR_TILE_H
#define FR_TILE_H 8
#endif
// 8 rows (4 or 16 also work: one warp per 8 x 4 pixels); 16 x 4 tiles
// measured 5% slower in the forward (more, smaller CTAs) and 1% in the
// adjustment (more padding in the flame-ray runs), 16 x 16 tiles (with 3 CTAs
// per SM) 7% slower in the forward
constexpr int kTileH = FR_TILE_H;
constexpr int kTileThreads = kTileW * kTileH;
// flame-list entry that names no pixel (padding)
constexpr unsigned kNoPixel = 0xffffffffu;

// Camera in voxel coordinates.
struct CamDev {
    float o[3];          // pinhole
    float r[3], u[3], f[3];
    float tx, ty;        // tan(half fov) * aspect, tan(half fov)
    int W, H;
};
static_assert(sizeof(CamDev) == 64, "CamDev layout");

// One reconstruction problem as the kernels see it.
struct ProbDev {
    const void* vol;             // records the rays sample
    const CamDev* cams;          // ncam cameras (device memory; batched launches only)
    int nx, ny, nz;
    int ncam, W, H;
    int tiles_x, tiles_y;        // tiles per view
    const float* targets;        // prepared targets (image layout), nullable
    const int* bbox;             // ncam x 4, nullable
    float* rendered;             // image layout, nullable
    float* residual;             // image layout, nullable
    float* partials;             // 4 floats per CTA (squared-error partials), nullable
    float* dV;                   // nodes x 4 accumulator (adjust / backward)
    const float* img_in;         // adjust: residual; backward: d(loss)/d(pixel)
    const float* L_total;        // backward: rendered radiance
    float img_scale;             // multiplies img_in
    const float4* lut;           // colour-temperature table, lut_m rows {r,g,b,0}
    int lut_m;
    float lut_t0, lut_scale;     // u = (T - lut_t0) * lut_scale, lut_scale = (m-1)/(t1-t0)
    float step, alpha_l, alpha_d, tau, g_std, thresh;
    unsigned long long seed;
    int iteration;
    // 1: a flame ray's parts (FR_ADJ_SPLIT) divide the samples the
    // adjustment's box range over adj_box keeps instead of its whole chord
    // (set only where the adjustment skips by adj_occ; the forward computes
    // the same range to place the part boundaries)
    int split_box;
    // single-problem forward march: CTA b takes tile tile_order[b] (nullable: tile b)
    const unsigned* tile_order;
    unsigned long long* counter; // sample counter, nullable
    // batched launches only
    const unsigned* list;        // flame-ray list (linear pixel indices)
    const unsigned* list_count;  // its length (device)
    void* vol_rw;                // volume updated by the apply step
    long long nodes;
    float* sqerr;                // 4 floats per iteration
    int ntiles;
    int sq_slot;                 // error slot of the launch's first iteration
    // x-pair records: pair i = {record i, record of its +x neighbour}; when
    // set, the forward march gathers a cell's corners two at a time from it
    const void* pairs;
    // occupancy of the bricks of kBrick^3 cells (1 = some corner record of the brick is
    // non-zero); when set, the forward march skips empty bricks
    const unsigned char* occ;
    const unsigned* occ_box;     // box of the non-empty bricks (brick-table layout)
    // index of this problem's first view in its G(s) stream (views rendered
    // one problem at a time keep their own index)
    int view_base;
    // visual hull tags of this problem (batched hull clear): key points whose
    // tag differs from hull_full are held at 0
    const unsigned* hull;
    unsigned hull_full;
    // when set, the adjustment's iteration index is iteration + *iter_dev
    // (loops whose iterations are counted on the device)
    const int* iter_dev;
    // flame-ray list the forward march writes (when set): flame pixels
    // appended warp by warp at *flist_count (zero before the launch)
    unsigned* flist;
    unsigned* flist_count;
    // when set (with flist), every flame ray is listed once per part of its
    // samples (FR_ADJ_SPLIT parts): an entry's top two bits hold the part, and
    // the transmittance at the start of the part is stored at the same list
    // position here
    float* flist_tm;
    // when set (with flist), the residual of each listed flame ray, three
    // floats at its list position (every part's entry), which the adjustment
    // reads instead of the residual image
    float* flist_dl;
    // bricks holding a key point inside the visual hull; when set, the
    // adjustment skips the others (their key points' updates are discarded)
    const unsigned char* adj_occ;
    const unsigned* adj_box;     // box of those bricks
    int nbx, nby, nbz;           // bricks along x, y and z
    // batched launches with ray parts: per pixel, the transmittance at the
    // start of parts 1 .. FR_ADJ_SPLIT - 1 (part-major: [(j - 1) npix + pixel]),
    // written by the forward march for flame pixels; the flame-ray list then
    // holds one entry per part (the part in an entry's top two bits)
    float* tpart;
};

// Bricks of 4^3 cells: finer bricks follow the flame's surface more tightly
// (fewer samples evaluated) at the price of larger tables and more brick
// crossings; 4^3 measured faster than 8^3.
#ifndef FR_BRICK_SHIFT
#define FR_BRICK_SHIFT 2
#endif
constexpr int kBrickShift = FR_BRICK_SHIFT;   // log2 of the cells per brick edge
constexpr int kBrick = 1 << kBrickShift;      // cells per brick edge

// Bounds checks of the checked build (-DFR_CHECKED): an index outside [0, n)
// is recorded in the translation unit's check word (bit `code`) and replaced
// by 0, so the access stays inside its buffer; the normal build compiles the
// checks away.  Codes: 1 record gather, 2 update reduction, 4 pixel,
// 8 flame-ray list entry, 16 brick, 32 node of a volume pass.
#ifdef FR_CHECKED
static __device__ unsigned g_fr_check_word;
__device__ __forceinline__ long long fr_checked(long long i, long long n, unsigned code)
{
    if (i < 0 || i >= n) {
        atomicOr(&g_fr_check_word, code);
        return 0;
    }
    return i;
}
#define FR_CHK(i, n, code) fr_checked((long long)(i), (long long)(n), (code))
#else
#define FR_CHK(i, n, code) (i)
#endif

// ---------------------------------------------------------------------------
// Rays
// ---------------------------------------------------------------------------

struct Ray {
    float p0x, p0y, p0z;   // box entry point (voxel coordinates)
    float dx, dy, dz;      // unit direction
    float idx, idy, idz;   // 1 / direction (infinite along an axis the ray does not move on)
    float chord;           // length inside the box
    int n;                 // number of segments
};

// Pinhole ray of pixel (px, py) clipped to the node box [0, n-1]^3; returns
// false when the ray misses it (or only grazes it).
__device__ __forceinline__ bool make_ray(const CamDev& c, int px, int py, int nx, int ny, int nz,
                                         float step, Ray& R)
{
    float a = (2.0f * (px + 0.5f) / (float)c.W - 1.0f) * c.tx;
    float b = (1.0f - 2.0f * (py + 0.5f) / (float)c.H) * c.ty;
    float dx = c.f[0] + a * c.r[0] + b * c.u[0];
    float dy = c.f[1] + a * c.r[1] + b * c.u[1];
    float dz = c.f[2] + a * c.r[2] + b * c.u[2];
    float inv = 1.0f / sqrtf(dx * dx + dy * dy + dz * dz);
    dx *= inv; dy *= inv; dz *= inv;
    float o[3] = {c.o[0], c.o[1], c.o[2]};
    float d[3] = {dx, dy, dz};
    // The entry point and chord come from correctly rounded quotients: they
    // fix the sample positions, hence each sample's cell and key points
    // (Eq. 10), and a sample within rounding of a cell face may land on
    // either side (products by the reciprocals would widen that window to
    // about 1.5 ulp).  The reciprocals serve the brick and box clipping,
    // whose 1e-3 voxel margins absorb their rounding.
    float id[3] = {1.0f / dx, 1.0f / dy, 1.0f / dz};
    float hi[3] = {(float)(nx - 1), (float)(ny - 1), (float)(nz - 1)};
    float tin = -INFINITY, tout = INFINITY;
#pragma unroll
    for (int ax = 0; ax < 3; ++ax) {
        if (d[ax] == 0.0f) {
            if (o[ax] < 0.0f || o[ax] > hi[ax]) return false;
            continue;
        }
        float t0 = (0.0f - o[ax]) / d[ax];
        float t1 = (hi[ax] - o[ax]) / d[ax];
        tin = fmaxf(tin, fminf(t0, t1));
        tout = fminf(tout, fmaxf(t0, t1));
    }
    tin = fmaxf(tin, 0.0f);
    if (!(tout > tin)) return false;
    R.p0x = o[0] + tin * dx;
    R.p0y = o[1] + tin * dy;
    R.p0z = o[2] + tin * dz;
    R.dx = dx; R.dy = dy; R.dz = dz;
    R.idx = id[0]; R.idy = id[1]; R.idz = id[2];
    R.chord = tout - tin;
    R.n = (int)ceilf(R.chord / step);
    return R.n > 0;
}

// Segment k of a ray: its length and midpoint.
__device__ __forceinline__ void segment(const Ray& R, float step, int k, float& len,
                                        float& x, float& y, float& z)
{
    float ta = (float)k * step;
    float tb = fminf(ta + step, R.chord);
    len = tb - ta;
    float tm = 0.5f * (ta + tb);
    x = fmaf(tm, R.dx, R.p0x);
    y = fmaf(tm, R.dy, R.p0y);
    z = fmaf(tm, R.dz, R.p0z);
}

// Cell index clamped to [0, n-2] and the fraction inside it.  Sample points
// lie on the clipped chord, so the fraction is in [0, 1] up to rounding; the
// clamp keeps every index inside the volume whatever the input.
__device__ __forceinline__ void locate(float p, int n, int& i, float& f)
{
    const int ii = min(max(__float2int_rd(p), 0), n - 2);
    i = ii;
    f = p - (float)ii;
}

struct Cell {
    long long base;      // index of the lower corner
    float fx, fy, fz;
};

__device__ __forceinline__ Cell cell_of(float x, float y, float z, int nx, int ny, int nz)
{
    Cell c;
    int i, j, k;
    locate(x, nx, i, c.fx);
    locate(y, ny, j, c.fy);
    locate(z, nz, k, c.fz);
    c.base = ((long long)k * ny + j) * nx + i;
    return c;
}

// Cell indices of a sample (clamped as in cell_of) and its fractions.
struct CellIJK {
    int i, j, k;
    float fx, fy, fz;
};

__device__ __forceinline__ CellIJK cell_ijk(float x, float y, float z, int nx, int ny, int nz)
{
    CellIJK c;
    locate(x, nx, c.i, c.fx);
    locate(y, ny, c.j, c.fy);
    locate(z, nz, c.k, c.fz);
    return c;
}

// A ray's window on the eight key points of the cell it is in.  Slot t holds
// the key point whose node coordinates have parities (t & 1, (t >> 1) & 1,
// t >> 2).  When the ray moves to another cell, a key point shared by both
// cells keeps its slot, so only the slots whose key point changes are
// released (leave) and refilled (enter).  Every slot is visited on every move
// under its own predicate, so lanes of a warp that move differently run the
// same instructions.  Trilinear weights and key-point distances of slot t are
// the usual ones written with the fraction mirrored where the cell index is
// odd (mirror_frac).
struct Win {
    int base;                // node index of the cell's lowest corner; volumes hold < 2^31 nodes
    int nd[8];               // node held by slot t
    bool live;
};

// Nodes of the eight slots for the cell whose lowest corner is node `base` at
// (i, j, k): slot bit value v along an axis names node c + (v ^ (c & 1)).
__device__ __forceinline__ void win_nodes(int base, int i, int j, int k, int nx, int nxy, int nd[8])
{
    const int px = i & 1, py = j & 1, pz = k & 1;
    const int ox0 = px, ox1 = 1 - px;
    const int oy0 = py ? nx : 0, oy1 = py ? 0 : nx;
    const int zb0 = base + (pz ? nxy : 0), zb1 = base + (pz ? 0 : nxy);
    const int xy[4] = {ox0 + oy0, ox1 + oy0, ox0 + oy1, ox1 + oy1};
#pragma unroll
    for (int t = 0; t < 8; ++t) nd[t] = ((t >> 2) ? zb1 : zb0) + xy[t & 3];
}

// Move the window to cell (i, j, k).  leave(t, node, p) and then
// enter(t, node, p) run for every slot, p telling whether the slot's key point
// changes (leave with its old node, enter with its new one); the callbacks
// predicate their memory operations on p.  On the first call every slot
// enters.  A key point shared by both cells has the same parities in both, so
// it keeps its slot.  No branch depends on the cell: a warp's lanes, which
// enter cells at different samples, stay converged (the adjustment measured
// 3.7% faster than with a branch on the cell change and 2.6% more than with a
// branch per slot).
template <class Leave, class Enter>
__device__ __forceinline__ void win_move_pred(Win& W, int i, int j, int k, int nx, int ny, int nxy, Leave&& leave,
                                              Enter&& enter)
{
    const int base = (k * ny + j) * nx + i;
    int nn[8];
    win_nodes(base, i, j, k, nx, nxy, nn);
    W.base = base;
    const bool first = !W.live;
    W.live = true;
#pragma unroll
    for (int t = 0; t < 8; ++t) {
        const bool go = first || nn[t] != W.nd[t];
        leave(t, first ? nn[t] : W.nd[t], go && !first);   // (a valid node even when nothing leaves)
        W.nd[t] = nn[t];
        enter(t, nn[t], go);
    }
}

template <class Leave>
__device__ __forceinline__ void win_release(const Win& W, Leave&& leave)
{
    if (!W.live) return;
#pragma unroll
    for (int t = 0; t < 8; ++t) leave(t, W.nd[t]);
}

// Fraction toward the odd-parity key point along one axis.  (|f - (cell & 1)|,
// the same value, measured slower in the adjustment.)
__device__ __forceinline__ float mirror_frac(int cell, float f) { return (cell & 1) ? 1.0f - f : f; }

// 2^x on the special-function unit (flush-to-zero, about 2 ulp).
__device__ __forceinline__ float ex2_approx(float x)
{
    float y;
    asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}

// log2(e), to write exp(x) as 2^(x log2 e)
constexpr float kLog2e = 1.4426950408889634f;

// exp(-a |x|) for x = squared distance, given c = -a log2(e); the square
// root on the special-function unit (x = 0 gives 0; measured 2% faster than
// x rsqrt(x) with its guard against x = 0).
__device__ __forceinline__ float dist_weight(float c, float x)
{
    float r;
    asm("sqrt.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
    return ex2_approx(c * r);
}

// ---------------------------------------------------------------------------
// Node records
// ---------------------------------------------------------------------------

__device__ __forceinline__ float bf16_lo(uint32_t v) { return __uint_as_float(v << 16); }
__device__ __forceinline__ float bf16_hi(uint32_t v) { return __uint_as_float(v & 0xffff0000u); }

__device__ __forceinline__ float2 f16x2(uint32_t v)
{
    __half2 h = *reinterpret_cast<__half2*>(&v);
    return __half22float2(h);
}

// RGB record {S_r, S_g, S_b, sigma} of node `idx`.
template <int DT>
__device__ __forceinline__ float4 load_rgb(const void* vol, long long idx)
{
    if constexpr (DT == DT_F32) {
        return __ldg(reinterpret_cast<const float4*>(vol) + idx);
    } else {
        uint2 u = __ldg(reinterpret_cast<const uint2*>(vol) + idx);
        if constexpr (DT == DT_BF16) {
            return make_float4(bf16_lo(u.x), bf16_hi(u.x), bf16_lo(u.y), bf16_hi(u.y));
        } else {
            float2 a = f16x2(u.x), b = f16x2(u.y);
            return make_float4(a.x, a.y, b.x, b.y);
        }
    }
}

// sigma of an RGB record.
template <int DT>
__device__ __forceinline__ float load_rgb_sigma(const void* vol, long long idx)
{
    if constexpr (DT == DT_F32) {
        return __ldg(reinterpret_cast<const float*>(vol) + 4 * idx + 3);
    } else if constexpr (DT == DT_BF16) {
        return __uint_as_float((uint32_t)__ldg(reinterpret_cast<const unsigned short*>(vol) + 4 * idx + 3) << 16);
    } else {
        unsigned short h = __ldg(reinterpret_cast<const unsigned short*>(vol) + 4 * idx + 3);
        return __half2float(__ushort_as_half(h));
    }
}

// Temperature record {T, sigma}.
template <int DT>
__device__ __forceinline__ float2 load_ts(const void* vol, long long idx)
{
    if constexpr (DT == DT_F32) {
        return __ldg(reinterpret_cast<const float2*>(vol) + idx);
    } else {
        uint32_t u = __ldg(reinterpret_cast<const unsigned int*>(vol) + idx);
        if constexpr (DT == DT_BF16) return make_float2(bf16_lo(u), bf16_hi(u));
        else return f16x2(u);
    }
}

template <int DT>
__device__ __forceinline__ void store_rgb(void* vol, long long idx, float4 v)
{
    if constexpr (DT == DT_F32) {
        reinterpret_cast<float4*>(vol)[idx] = v;
    } else if constexpr (DT == DT_BF16) {
        __nv_bfloat162 a = __floats2bfloat162_rn(v.x, v.y), b = __floats2bfloat162_rn(v.z, v.w);
        uint2 u;
        u.x = *reinterpret_cast<uint32_t*>(&a);
        u.y = *reinterpret_cast<uint32_t*>(&b);
        reinterpret_cast<uint2*>(vol)[idx] = u;
    } else {
        __half2 a = __floats2half2_rn(v.x, v.y), b = __floats2half2_rn(v.z, v.w);
        uint2 u;
        u.x = *reinterpret_cast<uint32_t*>(&a);
        u.y = *reinterpret_cast<uint32_t*>(&b);
        reinterpret_cast<uint2*>(vol)[idx] = u;
    }
}

template <int DT>
__device__ __forceinline__ void store_ts(void* vol, long long idx, float2 v)
{
    if constexpr (DT == DT_F32) {
        reinterpret_cast<float2*>(vol)[idx] = v;
    } else if constexpr (DT == DT_BF16) {
        __nv_bfloat162 a = __floats2bfloat162_rn(v.x, v.y);
        reinterpret_cast<__nv_bfloat162*>(vol)[idx] = a;
    } else {
        reinterpret_cast<__half2*>(vol)[idx] = __floats2half2_rn(v.x, v.y);
    }
}

// x-pair records (record i and its +x neighbour, adjacent in memory).
// The FP32 x-pair record load of load_rgb_pair when need != 0; a and b keep
// their values otherwise (one predicated load, no branch).
__device__ __forceinline__ void load_rgb_pair_f32_if(const void* pairs, long long idx, unsigned need, float4& a,
                                                     float4& b)
{
    const float* p = reinterpret_cast<const float*>(pairs) + 8 * idx;
    asm("{\n\t.reg .pred q;\n\tsetp.ne.u32 q, %9, 0;\n\t"
        "@q ld.global.nc.v8.f32 {%0, %1, %2, %3, %4, %5, %6, %7}, [%8];\n\t}"
        : "+f"(a.x), "+f"(a.y), "+f"(a.z), "+f"(a.w), "+f"(b.x), "+f"(b.y), "+f"(b.z), "+f"(b.w)
        : "l"(p), "r"(need));
}

template <int DT>
__device__ __forceinline__ void load_rgb_pair(const void* pairs, long long idx, float4& a, float4& b)
{
    if constexpr (DT == DT_F32) {
        const float* p = reinterpret_cast<const float*>(pairs) + 8 * idx;
        asm("ld.global.nc.v8.f32 {%0, %1, %2, %3, %4, %5, %6, %7}, [%8];"
            : "=f"(a.x), "=f"(a.y), "=f"(a.z), "=f"(a.w), "=f"(b.x), "=f"(b.y), "=f"(b.z), "=f"(b.w)
            : "l"(p));
    } else {
        const uint4 u = __ldg(reinterpret_cast<const uint4*>(pairs) + idx);
        if constexpr (DT == DT_BF16) {
            a = make_float4(bf16_lo(u.x), bf16_hi(u.x), bf16_lo(u.y), bf16_hi(u.y));
            b = make_float4(bf16_lo(u.z), bf16_hi(u.z), bf16_lo(u.w), bf16_hi(u.w));
        } else {
            const float2 a0 = f16x2(u.x), a1 = f16x2(u.y), b0 = f16x2(u.z), b1 = f16x2(u.w);
            a = make_float4(a0.x, a0.y, a1.x, a1.y);
            b = make_float4(b0.x, b0.y, b1.x, b1.y);
        }
    }
}

template <int DT>
__device__ __forceinline__ void load_ts_pair(const void* pairs, long long idx, float2& a, float2& b)
{
    if constexpr (DT == DT_F32) {
        const float4 f = __ldg(reinterpret_cast<const float4*>(pairs) + idx);
        a = make_float2(f.x, f.y);
        b = make_float2(f.z, f.w);
    } else {
        const uint2 u = __ldg(reinterpret_cast<const uint2*>(pairs) + idx);
        if constexpr (DT == DT_BF16) {
            a = make_float2(bf16_lo(u.x), bf16_hi(u.x));
            b = make_float2(bf16_lo(u.y), bf16_hi(u.y));
        } else {
            a = f16x2(u.x);
            b = f16x2(u.y);
        }
    }
}

__device__ __forceinline__ float lerpf(float a, float b, float t) { return fmaf(t, b - a, a); }

// Packed FP32 pairs: sm_100-family GPUs execute add/sub/mul/fma on two floats
// held in a 64-bit register pair as one instruction (.f32x2), each half
// rounded to nearest exactly as the scalar operation.  Used for the
// trilinear blends and the adjustment's distance weights: the forward march
// measured 6.5% faster (0.268 against 0.287 ms on the 128^3 x 8 x 512^2
// step), the adjustment 0.5%.  FR_PACKED = 0 keeps the scalar forms.
#ifndef FR_PACKED
#define FR_PACKED 1
#endif
struct F2 {
    unsigned long long v;
};
__device__ __forceinline__ F2 f2(float lo, float hi)
{
    F2 r;
    asm("mov.b64 %0, {%1, %2};" : "=l"(r.v) : "f"(lo), "f"(hi));
    return r;
}
__device__ __forceinline__ float2 f2_get(F2 a)
{
    float2 r;
    asm("mov.b64 {%0, %1}, %2;" : "=f"(r.x), "=f"(r.y) : "l"(a.v));
    return r;
}
__device__ __forceinline__ F2 f2_add(F2 a, F2 b)
{
    F2 r;
    asm("add.rn.f32x2 %0, %1, %2;" : "=l"(r.v) : "l"(a.v), "l"(b.v));
    return r;
}
__device__ __forceinline__ F2 f2_sub(F2 a, F2 b)
{
    F2 r;
    asm("sub.rn.f32x2 %0, %1, %2;" : "=l"(r.v) : "l"(a.v), "l"(b.v));
    return r;
}
__device__ __forceinline__ F2 f2_mul(F2 a, F2 b)
{
    F2 r;
    asm("mul.rn.f32x2 %0, %1, %2;" : "=l"(r.v) : "l"(a.v), "l"(b.v));
    return r;
}
__device__ __forceinline__ F2 f2_fma(F2 a, F2 b, F2 c)
{
    F2 r;
    asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(r.v) : "l"(a.v), "l"(b.v), "l"(c.v));
    return r;
}
// lerpf on both halves with one weight t (the same two roundings per half)
__device__ __forceinline__ F2 f2_lerp(F2 a, F2 b, F2 t) { return f2_fma(t, f2_sub(b, a), a); }

__device__ __forceinline__ float4 lerp4(float4 a, float4 b, float t)
{
#if FR_PACKED
    const F2 tt = f2(t, t);
    const float2 lo = f2_get(f2_lerp(f2(a.x, a.y), f2(b.x, b.y), tt));
    const float2 hi = f2_get(f2_lerp(f2(a.z, a.w), f2(b.z, b.w), tt));
    return make_float4(lo.x, lo.y, hi.x, hi.y);
#else
    return make_float4(lerpf(a.x, b.x, t), lerpf(a.y, b.y, t), lerpf(a.z, b.z, t), lerpf(a.w, b.w, t));
#endif
}

__device__ __forceinline__ float2 lerp2(float2 a, float2 b, float t)
{
    return make_float2(lerpf(a.x, b.x, t), lerpf(a.y, b.y, t));
}

// Trilinear blend of the eight RGB records around a sample.
template <int DT>
__device__ __forceinline__ float4 sample_rgb(const void* vol, const Cell& c, int nx, long long nxy)
{
    const long long b = c.base;
    float4 v000 = load_rgb<DT>(vol, b), v100 = load_rgb<DT>(vol, b + 1);
    float4 v010 = load_rgb<DT>(vol, b + nx), v110 = load_rgb<DT>(vol, b + nx + 1);
    float4 v001 = load_rgb<DT>(vol, b + nxy), v101 = load_rgb<DT>(vol, b + nxy + 1);
    float4 v011 = load_rgb<DT>(vol, b + nxy + nx), v111 = load_rgb<DT>(vol, b + nxy + nx + 1);
    float4 c00 = lerp4(v000, v100, c.fx), c10 = lerp4(v010, v110, c.fx);
    float4 c01 = lerp4(v001, v101, c.fx), c11 = lerp4(v011, v111, c.fx);
    return lerp4(lerp4(c00, c10, c.fy), lerp4(c01, c11, c.fy), c.fz);
}

template <int DT>
__device__ __forceinline__ float sample_rgb_sigma(const void* vol, const Cell& c, int nx, long long nxy)
{
    const long long b = c.base;
    float s000 = load_rgb_sigma<DT>(vol, b), s100 = load_rgb_sigma<DT>(vol, b + 1);
    float s010 = load_rgb_sigma<DT>(vol, b + nx), s110 = load_rgb_sigma<DT>(vol, b + nx + 1);
    float s001 = load_rgb_sigma<DT>(vol, b + nxy), s101 = load_rgb_sigma<DT>(vol, b + nxy + 1);
    float s011 = load_rgb_sigma<DT>(vol, b + nxy + nx), s111 = load_rgb_sigma<DT>(vol, b + nxy + nx + 1);
    float c00 = lerpf(s000, s100, c.fx), c10 = lerpf(s010, s110, c.fx);
    float c01 = lerpf(s001, s101, c.fx), c11 = lerpf(s011, s111, c.fx);
    return lerpf(lerpf(c00, c10, c.fy), lerpf(c01, c11, c.fy), c.fz);
}

template <int DT>
__device__ __forceinline__ float2 sample_ts(const void* vol, const Cell& c, int nx, long long nxy)
{
    const long long b = c.base;
    float2 v000 = load_ts<DT>(vol, b), v100 = load_ts<DT>(vol, b + 1);
    float2 v010 = load_ts<DT>(vol, b + nx), v110 = load_ts<DT>(vol, b + nx + 1);
    float2 v001 = load_ts<DT>(vol, b + nxy), v101 = load_ts<DT>(vol, b + nxy + 1);
    float2 v011 = load_ts<DT>(vol, b + nxy + nx), v111 = load_ts<DT>(vol, b + nxy + nx + 1);
    float2 c00 = lerp2(v000, v100, c.fx), c10 = lerp2(v010, v110, c.fx);
    float2 c01 = lerp2(v001, v101, c.fx), c11 = lerp2(v011, v111, c.fx);
    return lerp2(lerp2(c00, c10, c.fy), lerp2(c01, c11, c.fy), c.fz);
}

// Piecewise-linear colour-temperature lookup and the slope of that
// interpolant (zero outside the table, where the value is clamped).
__device__ __forceinline__ void lut_eval(const ProbDev& P, float T, float q[3], float dq[3])
{
    float u = (T - P.lut_t0) * P.lut_scale;
    const float umax = (float)(P.lut_m - 1);
    bool inside = (u >= 0.0f) && (u <= umax);
    u = fminf(fmaxf(u, 0.0f), umax);
    int i = min((int)u, P.lut_m - 2);
    float f = u - (float)i;
    float4 a = __ldg(P.lut + i), b = __ldg(P.lut + i + 1);
    q[0] = lerpf(a.x, b.x, f);
    q[1] = lerpf(a.y, b.y, f);
    q[2] = lerpf(a.z, b.z, f);
    float s = inside ? P.lut_scale : 0.0f;
    dq[0] = (b.x - a.x) * s;
    dq[1] = (b.y - a.y) * s;
    dq[2] = (b.z - a.z) * s;
}

// (1 - exp(-a)) / sigma for a = sigma * len, given e = exp(-a); a Taylor
// series near a = 0 avoids the cancellation in 1 - e.
// FR_SEG_SELECT = 1: no branch (the in-scattering sweeps measured 8.5%
// faster, 0.062 against 0.068 ms at 128^3; the forward march the same)
#ifndef FR_SEG_SELECT
#define FR_SEG_SELECT 1
#endif
__device__ __forceinline__ float seg_weight(float sig, float len, float e)
{
    float a = sig * len;
#if FR_SEG_SELECT
    // both forms and a select, no branch (a warp's lanes take different
    // ones); the quotient with the approximate reciprocal (2 ulp)
    const float series =
        len * (1.0f - a * (0.5f - a * (1.0f / 6.0f - a * (1.0f / 24.0f - a * (1.0f / 120.0f - a * (1.0f / 720.0f))))));
    const float quot = __fdividef(1.0f - e, sig);
    return fabsf(a) < 0.1f ? series : quot;
#else
    if (fabsf(a) < 0.1f) {
        return len * (1.0f - a * (0.5f - a * (1.0f / 6.0f - a * (1.0f / 24.0f - a * (1.0f / 120.0f - a * (1.0f / 720.0f))))));
    }
    return (1.0f - e) / sig;
#endif
}

// d/dsigma of seg_weight.
__device__ __forceinline__ float seg_weight_dsigma(float sig, float len, float e, float beta)
{
    float a = sig * len;
    if (fabsf(a) < 0.1f) {
        return -len * len * (0.5f - a * (1.0f / 3.0f - a * (1.0f / 8.0f - a * (1.0f / 30.0f - a * (1.0f / 144.0f)))));
    }
    return (len * e - beta) / sig;
}

// ---------------------------------------------------------------------------
// G(s) of Eq. 11: outputs 2c+1 and 2c+2 of the SplitMix64 sequence started at
// `seed` (Steele, Lea and Flood, OOPSLA 2014), c = (iteration, view, pixel,
// sample) packed in 64 bits, made Gaussian by the Box-Muller transform.
// ---------------------------------------------------------------------------

__device__ __forceinline__ unsigned long long splitmix_out(unsigned long long seed, unsigned long long n)
{
    unsigned long long z = seed + n * 0x9E3779B97F4A7C15ull;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

__device__ __forceinline__ float g_draw(unsigned long long seed, float g_std, int iteration, int view,
                                        int pixel, int k)
{
    unsigned long long c = ((unsigned long long)iteration << 44) | ((unsigned long long)view << 36) |
                           ((unsigned long long)pixel << 14) | (unsigned long long)k;
    unsigned long long r1 = splitmix_out(seed, 2 * c + 1), r2 = splitmix_out(seed, 2 * c + 2);
    float u1 = ((float)(r1 >> 40) + 0.5f) * (1.0f / 16777216.0f);
    float u2 = (float)(r2 >> 40) * (1.0f / 16777216.0f);
    return 1.0f + g_std * sqrtf(-2.0f * logf(u1)) * cospif(2.0f * u2);
}

// ---------------------------------------------------------------------------
// Reductions
// ---------------------------------------------------------------------------

__device__ __forceinline__ void red_add_v4(float* addr, float a, float b, float c, float d)
{
    asm volatile("red.global.add.v4.f32 [%0], {%1, %2, %3, %4};"
                 :: "l"(addr), "f"(a), "f"(b), "f"(c), "f"(d) : "memory");
}

__device__ __forceinline__ void red_add_v2(float* addr, float a, float b)
{
    asm volatile("red.global.add.v2.f32 [%0], {%1, %2};" :: "l"(addr), "f"(a), "f"(b) : "memory");
}

__device__ __forceinline__ void red_add_v4_if(float* addr, float a, float b, float c, float d, bool p)
{
    asm volatile("{\n\t.reg .pred q;\n\tsetp.ne.u32 q, %5, 0;\n\t"
                 "@q red.global.add.v4.f32 [%0], {%1, %2, %3, %4};\n\t}"
                 :: "l"(addr), "f"(a), "f"(b), "f"(c), "f"(d), "r"((unsigned)p) : "memory");
}

__device__ __forceinline__ void red_add_v2_if(float* addr, float a, float b, bool p)
{
    asm volatile("{\n\t.reg .pred q;\n\tsetp.ne.u32 q, %3, 0;\n\t@q red.global.add.v2.f32 [%0], {%1, %2};\n\t}"
                 :: "l"(addr), "f"(a), "f"(b), "r"((unsigned)p) : "memory");
}

__device__ __forceinline__ void load_f32_if(const float* addr, bool p, float& v)
{
    asm("{\n\t.reg .pred q;\n\tsetp.ne.u32 q, %2, 0;\n\t@q ld.global.nc.f32 %0, [%1];\n\t}"
        : "+f"(v) : "l"(addr), "r"((unsigned)p));
}

// A BF16 value loaded and widened to FP32 when p (v kept otherwise).
__device__ __forceinline__ void load_bf16_if(const unsigned short* addr, bool p, float& v)
{
    asm("{\n\t.reg .pred q;\n\t.reg .b32 r;\n\tsetp.ne.u32 q, %2, 0;\n\t"
        "@q ld.global.nc.u16 r, [%1];\n\t@q shl.b32 r, r, 16;\n\t@q mov.b32 %0, r;\n\t}"
        : "+f"(v) : "l"(addr), "r"((unsigned)p));
}

// An FP16 value loaded and widened to FP32 when p (v kept otherwise).
__device__ __forceinline__ void load_f16_if(const unsigned short* addr, bool p, float& v)
{
    asm("{\n\t.reg .pred q;\n\t.reg .b16 h;\n\tsetp.ne.u32 q, %2, 0;\n\t"
        "@q ld.global.nc.b16 h, [%1];\n\t@q cvt.f32.f16 %0, h;\n\t}"
        : "+f"(v) : "l"(addr), "r"((unsigned)p));
}

__device__ __forceinline__ float warp_sum(float v)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// The error sums of one pass over nb CTAs of up to 256 threads: CTA b sums
// its share of the tiles' partials (float4 per tile) into part_sums[b]; the
// last CTA to finish (counted in *done, which it resets to 0) adds the shares
// in order, so the result does not depend on which CTA ends last, writes
// out4 (added to it when accumulate) and, with rmse3, the error measure of
// Sec. 5.1, 255 sqrt(sum / count) per channel.
__device__ __forceinline__ void finalize_parts_body(const float* __restrict__ partials, int ntiles,
                                                    float* __restrict__ out4, int accumulate, float4* part_sums,
                                                    unsigned* done, float* rmse3, unsigned b, unsigned nb)
{
    __shared__ float red[4][8];
    __shared__ bool last;
    __shared__ float sum4[4];
    const int per = (ntiles + (int)nb - 1) / (int)nb;
    const int b0 = (int)b * per, b1 = min(b0 + per, ntiles);
    float s0 = 0.0f, s1 = 0.0f, s2 = 0.0f, s3 = 0.0f;
    const float4* p4 = reinterpret_cast<const float4*>(partials);
#pragma unroll 4
    for (int i = b0 + threadIdx.x; i < b1; i += blockDim.x) {
        const float4 v = __ldg(p4 + i);
        s0 += v.x; s1 += v.y; s2 += v.z; s3 += v.w;
    }
    s0 = warp_sum(s0); s1 = warp_sum(s1); s2 = warp_sum(s2); s3 = warp_sum(s3);
    const int w = threadIdx.x >> 5;
    if ((threadIdx.x & 31) == 0) { red[0][w] = s0; red[1][w] = s1; red[2][w] = s2; red[3][w] = s3; }
    __syncthreads();
    if (threadIdx.x == 0) {
        float4 t = make_float4(0.0f, 0.0f, 0.0f, 0.0f);
        for (int i = 0; i < (int)(blockDim.x >> 5); ++i) {
            t.x += red[0][i]; t.y += red[1][i]; t.z += red[2][i]; t.w += red[3][i];
        }
        part_sums[b] = t;
        __threadfence();
        last = atomicAdd(done, 1u) == nb - 1;
    }
    __syncthreads();
    if (!last) return;
    if (threadIdx.x < 4) {
        __threadfence();
        const volatile float* ps = reinterpret_cast<const volatile float*>(part_sums);
        float t = 0.0f;
        for (int i = 0; i < (int)nb; ++i) t += ps[4 * i + threadIdx.x];
        t = accumulate ? out4[threadIdx.x] + t : t;
        out4[threadIdx.x] = t;
        sum4[threadIdx.x] = t;
    }
    if (threadIdx.x == 0) *done = 0u;
    if (rmse3) {
        __syncthreads();
        if (threadIdx.x < 3) {
            const float cnt = sum4[3];
            rmse3[threadIdx.x] = cnt > 0.0f ? 255.0f * sqrtf(sum4[threadIdx.x] / cnt) : 0.0f;
        }
    }
}

// View and pixel of the calling thread's ray in CTA tile `tile`.
__device__ __forceinline__ void tile_pixel(const ProbDev& P, int tile, int& view, int& px, int& py)
{
    const int per_view = P.tiles_x * P.tiles_y;
    view = tile / per_view;
    const int t = tile - view * per_view;
    const int ty = t / P.tiles_x, tx = t - ty * P.tiles_x;
    const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
    px = tx * kTileW + (w & 1) * 8 + (lane & 7);
    py = ty * kTileH + (w >> 1) * 4 + (lane >> 3);
}

__device__ __forceinline__ int find_problem(const int* __restrict__ tile_start, int nprob, int b)
{
    int lo = 0, hi = nprob - 1;
    while (lo < hi) {
        int mid = (lo + hi + 1) >> 1;
        if (__ldg(tile_start + mid) <= b) lo = mid; else hi = mid - 1;
    }
    return lo;
}

// Trilinear blend of eight parity slots with mirrored fractions gx, gy, gz.
template <class R>
__device__ __forceinline__ R slot_blend(const R* v, float gx, float gy, float gz);

template <>
__device__ __forceinline__ float4 slot_blend<float4>(const float4* v, float gx, float gy, float gz)
{
    float4 a = lerp4(v[0], v[1], gx), b = lerp4(v[2], v[3], gx);
    float4 c = lerp4(v[4], v[5], gx), d = lerp4(v[6], v[7], gx);
    return lerp4(lerp4(a, b, gy), lerp4(c, d, gy), gz);
}

template <>
__device__ __forceinline__ float2 slot_blend<float2>(const float2* v, float gx, float gy, float gz)
{
    float2 a = lerp2(v[0], v[1], gx), b = lerp2(v[2], v[3], gx);
    float2 c = lerp2(v[4], v[5], gx), d = lerp2(v[6], v[7], gx);
    return lerp2(lerp2(a, b, gy), lerp2(c, d, gy), gz);
}

template <>
__device__ __forceinline__ float slot_blend<float>(const float* v, float gx, float gy, float gz)
{
#if FR_PACKED
    // the same lerps, slots t and t + 4 side by side: (a, c), (b, d), then
    // (lerp(a, b), lerp(c, d)) and the z lerp
    const F2 tx = f2(gx, gx), ty = f2(gy, gy);
    const F2 ac = f2_lerp(f2(v[0], v[4]), f2(v[1], v[5]), tx);
    const F2 bd = f2_lerp(f2(v[2], v[6]), f2(v[3], v[7]), tx);
    const float2 e = f2_get(f2_lerp(ac, bd, ty));
    return lerpf(e.x, e.y, gz);
#else
    float a = lerpf(v[0], v[1], gx), b = lerpf(v[2], v[3], gx);
    float c = lerpf(v[4], v[5], gx), d = lerpf(v[6], v[7], gx);
    return lerpf(lerpf(a, b, gy), lerpf(c, d, gy), gz);
#endif
}

// Skipping of flagged-off bricks along one ray.  A brick is the box of kBrick^3
// cells [B b, min(B b + B, n - 1)] per axis (B = kBrick); `flags` holds one byte per brick
// (non-zero: the samples in it are evaluated).
struct BrickSkip {
    int brick = -1;         // the brick of the last tested sample
    bool occupied = true;   // and its flag

    // Samples [k0, k1) of the ray that can lie in the box of the flagged-on
    // bricks (box: brick-table layout); false when there are none.  Samples
    // outside the range have their midpoint (their start, for the last,
    // shorter segment) beyond the box by more than a 1e-3 voxel margin.
    static __device__ __forceinline__ bool box_range(const ProbDev& P, const unsigned* box, const Ray& R,
                                                     float step, int& k0, int& k1)
    {
        const unsigned hx = __ldg(box + 3), hy = __ldg(box + 4), hz = __ldg(box + 5);
        if (hx == 0u) return false;
        const float lo[3] = {(float)((P.nbx - (int)__ldg(box)) * kBrick), (float)((P.nby - (int)__ldg(box + 1)) * kBrick),
                             (float)((P.nbz - (int)__ldg(box + 2)) * kBrick)};
        const float hi[3] = {(float)min((int)hx * kBrick, P.nx - 1), (float)min((int)hy * kBrick, P.ny - 1),
                             (float)min((int)hz * kBrick, P.nz - 1)};
        const float o[3] = {R.p0x, R.p0y, R.p0z}, d[3] = {R.dx, R.dy, R.dz}, id[3] = {R.idx, R.idy, R.idz};
        float tin = 0.0f, tout = R.chord;
#pragma unroll
        for (int a = 0; a < 3; ++a) {
            if (d[a] == 0.0f) {
                if (o[a] < lo[a] - 1e-3f || o[a] > hi[a] + 1e-3f) return false;
                continue;
            }
            const float t0 = (lo[a] - o[a]) * id[a], t1 = (hi[a] - o[a]) * id[a];
            tin = fmaxf(tin, fminf(t0, t1));
            tout = fminf(tout, fmaxf(t0, t1));
        }
        // (the 1e-3 voxel margins cover the rounding of the products by
        // 1 / step, a few ulp of at most a few hundred sample lengths)
        const float is = 1.0f / step;
        k0 = max(0, (int)ceilf((tin - 1e-3f) * is - 0.5f));
        k1 = min(R.n, (int)floorf((tout + 1e-3f) * is) + 1);
        return k0 < k1;
    }

    // True when sample k (midpoint x, y, z) lies in a flagged-off brick.  k
    // then moves so that the loop's increment lands on the first sample whose
    // midpoint may lie beyond that brick; a 1e-3 voxel margin on the exit
    // keeps rounding on the safe side.
    __device__ __forceinline__ bool empty(const unsigned char* flags, const ProbDev& P, const Ray& R, float step,
                                          float x, float y, float z, int& k)
    {
        return empty_at(flags, P, R, step, cell_ijk(x, y, z, P.nx, P.ny, P.nz), k);
    }

    // The same for the sample's cell c.
    __device__ __forceinline__ bool empty_at(const unsigned char* flags, const ProbDev& P, const Ray& R, float step,
                                             const CellIJK& c, int& k)
    {
        const int b = ((c.k >> kBrickShift) * P.nby + (c.j >> kBrickShift)) * P.nbx + (c.i >> kBrickShift);
        {
            // the flag reloaded by a predicated load when the brick changes
            // (no branch: 0.5-2% faster in the marches)
            unsigned f = occupied ? 1u : 0u;
            const unsigned need = b != brick ? 1u : 0u;
            const unsigned char* fp = flags + FR_CHK(b, (long long)P.nbx * P.nby * P.nbz, 16u);
            asm("{\n\t.reg .pred q;\n\tsetp.ne.u32 q, %2, 0;\n\t@q ld.global.nc.u8 %0, [%1];\n\t}"
                : "+r"(f) : "l"(fp), "r"(need));
            brick = b;
            occupied = f != 0u;
        }
        if (occupied) return false;
        const int bx = c.i & ~(kBrick - 1), by = c.j & ~(kBrick - 1), bz = c.k & ~(kBrick - 1);
        float te = INFINITY;
        if (R.dx != 0.0f) te = fminf(te, ((R.dx > 0.0f ? (float)min(bx + kBrick, P.nx - 1) : (float)bx) - R.p0x) * R.idx);
        if (R.dy != 0.0f) te = fminf(te, ((R.dy > 0.0f ? (float)min(by + kBrick, P.ny - 1) : (float)by) - R.p0y) * R.idy);
        if (R.dz != 0.0f) te = fminf(te, ((R.dz > 0.0f ? (float)min(bz + kBrick, P.nz - 1) : (float)bz) - R.p0z) * R.idz);
        const int kn = (int)ceilf((te - 1e-3f) / step - 0.5f);
        k = max(k, kn - 1);
        return true;
    }
};

}  // namespace frk
