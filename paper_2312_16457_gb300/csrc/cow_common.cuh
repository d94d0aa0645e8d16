// cow_common.cuh -- records and device helpers shared by the libcow kernels.
//
// Geometry decisions (which lattice samples exist, which block a sample falls
// in, which occupancy cell it lies in) are taken on FP32 values produced by a
// fixed sequence of IEEE round-to-nearest operations.  The __f*_rn intrinsics
// below keep nvcc from fusing or reordering them, so the decisions are a pure
// function of the inputs.
#pragma once

#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <cuda_fp8.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include <type_traits>

namespace cow {

constexpr int kNch = 8;
constexpr int kMlpParams = 499;
constexpr int kOffW1 = 0, kOffB1 = 160, kOffW2 = 176, kOffB2 = 432, kOffW3 = 448, kOffB3 = 496;
constexpr int kMaxRayIds = 64;       // blocks one ray of the ray-batch form composites
constexpr int kMaxSpan = 1 << 22;    // lattice indices one (ray, block) pair may scan

// error word bits (device-side faults are recorded, never trapped)
constexpr unsigned kErrRange = 1u;    // a (ray, block) candidate range exceeded kMaxSpan
constexpr unsigned kErrTimeout = 2u;  // a bounded wait ran out
constexpr unsigned kErrArg = 4u;      // a kernel met an argument it cannot handle

// kMixed: BF16 grid (pair layout) with FP8-E4M3 planes (quad layout: element
// (u, v) holds texels (u, v), (u+1, v), (u, v+1), (u+1, v+1), 8 bytes each).
// kFP8D: FP8-E4M3 features with the grid's log-density in BF16: the grid's
// eight channels in FP8 in the quad layout over (x, y) (element (x, y, z)
// holds vertices (x, y), (x+1, y), (x, y+1), (x+1, y+1) of slice z), channel
// 0 of the grid again in BF16 in the octet layout (element (x, y, z) holds
// the eight corners of voxel (x, y, z), corner k = dx + 2 dy + 4 dz, 16
// bytes), and the planes in FP8 in the quad layout.
enum Dtype { kF32 = 0, kF16 = 1, kBF16 = 2, kFP8 = 3, kMixed = 4, kFP8D = 5 };

// A kernel's DT template argument is the storage dtype, plus kBrickBit for a
// brick-sparse grid (its lookups go through the brick table; the dense
// variants keep the plain vertex indexing and register budget).
constexpr int kBrickBit = 8;
constexpr int kStoreMask = 7;

// Brick-sparse grids: the grid is cut into bricks of kBrick voxels per edge
// (one coarse occupancy cell, kOccGroup cells of 4 voxels); only bricks with
// an occupied cell are stored, each holding the elements of its voxels' first
// corners (with the layout's halo: 17 or 16 elements per axis).
constexpr int kBrickLog2 = 4;
constexpr int kBrick = 1 << kBrickLog2;
constexpr int kDensBrickElems = kBrick * kBrick * kBrick;  // kFP8D density octets per brick

// Unbounded boundary blocks (scene contraction, Eq. 16)
constexpr int kUnbXLo = 1, kUnbXHi = 2, kUnbYLo = 4, kUnbYHi = 8, kUnbContracted = 16;
constexpr float kContractMax = 1.0e4f;  // the march of an unbounded block stops beyond ||x||_inf = 1e4
constexpr int kContractSteps = 65536;   // and after this many steps

// Occupancy cells per coarse cell along each axis (the second level of the
// multi-level occupancy grid).
constexpr int kOccGroupLog2 = 2;
constexpr int kOccGroup = 1 << kOccGroupLog2;

// One block as the kernels see it (host fills it once at load time).
struct alignas(16) BlockRec {
    float lo[3], hi[3];      // world AABB (FP32, exactly the caller's values)
    float lo_e[3], hi_e[3];  // AABB grown by 1e-3 * max(1, extent): candidate-range box
    float kg[3];             // (float)((R-1) / (hi-lo)) per axis, computed in double
    float kp[3];             // (float)((P-1) / (hi-lo)) per axis, computed in double
    float delta;             // (float)((hi_x - lo_x) / P), computed in double
    float cx, cy;            // (float)((lo + hi) / 2) in double: ray-batch sort key
    float vox[3];            // (float)((hi-lo) / (R-1)): voxel pitch per axis
    float bmax;              // max |coordinate| of the box (scale of FP32 position error)
    int32_t R, P, Nc, C;     // resolutions, occupancy cells per axis, voxels per cell
    int32_t dtype;
    uint32_t cdiv;           // ceil(2^32 / C): v / C == umulhi(v, cdiv) for 0 <= v < 2^16, C >= 2
    const void *grid;        // packed R^3 x 8
    const void *planes[3];   // packed P^2 x 8 each (xy, xz, yz)
    const uint32_t *occ;     // occupancy bits
    const float *scale;      // 32 floats: per-channel scale of grid, xy, xz, yz
    const uint32_t *occ2;    // coarse occupancy: one bit per kOccGroup^3 cells (OR of their bits)
    int32_t Nc2;             // coarse cells per axis, ceil(Nc / kOccGroup)
    int32_t unb;             // 0, or kUnbContracted | the xy sides (kUnbX/YLo/Hi) extended to infinity
    float cc[3];             // unbounded: (float)((lo + hi) / 2), computed in double
    float ih[3];             // unbounded: (float)(2 / (hi - lo)), computed in double
    float plo[3];            // origin of the lookup coordinates: lo, or -2 (contracted u) when unbounded
    int32_t Nb;              // brick-sparse grid: bricks per axis (0 for a dense grid)
    const void *dens;        // kFP8D: BF16 log-density octets (dense: R^3 elements; bricks: 4096 a brick)
    const int32_t *brick;    // brick-sparse grid: slot of brick (bz, by, bx), -1 when not stored; null: dense
    int32_t bsy, bsz;        // element strides of the grid along y and z (dense: R, R^2; in a brick)
    int32_t belem;           // brick-sparse grid: elements per brick
    int32_t pad_;
    // when unbounded, kg and kp hold (R-1)/4 and (P-1)/4: lookups index u in [-2, 2]
};
static_assert(sizeof(BlockRec) % 16 == 0, "BlockRec must be a multiple of 16 bytes");
static_assert(sizeof(BlockRec) * 96 + 512 <= 32764, "96 records fit the kernel parameter space");
static_assert(sizeof(BlockRec) == 272, "BlockRec layout");

// The blocks of a ray-batch call (at most kMaxRayIds), passed by value in the
// launch's parameter buffer like ParamRecs: record k is block id[k].
struct RayRecs {
    BlockRec r[kMaxRayIds];
    int32_t id[kMaxRayIds];
    int32_t n;
    int32_t pad_[3];
};
static_assert(sizeof(RayRecs) + 512 <= 32764, "the ray-batch records fit the kernel parameter space");

// Block records passed by value in a launch's parameter buffer (a kernel's
// parameters may take up to 32764 bytes).
constexpr int kParamRecs = 96;
struct ParamRecs {
    BlockRec r[kParamRecs];
};

// One camera as the kernels see it.
struct alignas(16) ViewRec {
    float Rm[9];         // (float)c2w rotation, row-major
    float o[3];          // (float)c2w translation
    float f;             // (float)((H/2) / tan(fov/2)), computed in double
    int32_t W, H;
    int32_t tiles_x;     // tiles per image row
    int32_t tile_begin;  // first global tile index of this view
    int32_t ids_begin, ids_count;  // this view's block records: recs[ids_begin .. + ids_count)
    int32_t strip;                 // tile order: 0 raster, else vertical strips of `strip` tile columns
    int64_t pix_offset;  // first output row of this view
};
static_assert(sizeof(ViewRec) % 16 == 0, "ViewRec must be a multiple of 16 bytes");

// Tile t of a view -> tile coordinates.  Raster order, or vertical strips of
// v.strip tile columns walked row by row (the tiles in flight then cover a
// compact screen region instead of a full-width band of rows).
__device__ __forceinline__ void tile_xy(const ViewRec &v, int t, int tile_h, int &tx, int &ty) {
    if (v.strip <= 0 || v.strip >= v.tiles_x) {
        tx = t % v.tiles_x;
        ty = t / v.tiles_x;
        return;
    }
    const int tiles_y = (v.H + tile_h - 1) / tile_h;
    const int per_strip = v.strip * tiles_y;
    const int k = t / per_strip, r = t - k * per_strip;
    const int w = min(v.strip, v.tiles_x - k * v.strip);
    ty = r / w;
    tx = k * v.strip + (r - ty * w);
}

// ---------------------------------------------------------------------------
// FP32 decision sequence

// Pinhole ray through the centre of pixel (px, py).
__device__ __forceinline__ void pixel_ray(const ViewRec &v, int px, int py, float o[3], float d[3]) {
    const float bx = __fsub_rn(__fadd_rn((float)px, 0.5f), __fmul_rn(0.5f, (float)v.W));
    const float by = __fsub_rn(__fadd_rn((float)py, 0.5f), __fmul_rn(0.5f, (float)v.H));
    const float xc = __fdiv_rn(bx, v.f);
    const float yc = -__fdiv_rn(by, v.f);
    float dw[3];
#pragma unroll
    for (int r = 0; r < 3; r++) {
        const float s = __fadd_rn(__fmul_rn(v.Rm[3 * r + 0], xc), __fmul_rn(v.Rm[3 * r + 1], yc));
        dw[r] = __fsub_rn(s, v.Rm[3 * r + 2]);
        o[r] = v.o[r];
    }
    const float n2 =
        __fadd_rn(__fadd_rn(__fmul_rn(dw[0], dw[0]), __fmul_rn(dw[1], dw[1])), __fmul_rn(dw[2], dw[2]));
    const float n = __fsqrt_rn(n2);
#pragma unroll
    for (int r = 0; r < 3; r++) d[r] = __fdiv_rn(dw[r], n);
}

// Lattice sample i of a ray: t = (i + 1/2) delta, p = o + t d.
__device__ __forceinline__ void lattice_point(const float o[3], const float d[3], float delta, int i,
                                              float p[3]) {
    const float t = __fmul_rn(__fadd_rn(__int2float_rn(i), 0.5f), delta);
#pragma unroll
    for (int a = 0; a < 3; a++) p[a] = __fadd_rn(o[a], __fmul_rn(t, d[a]));
}

// Ground-plane membership: half-open in x and y, closed in z.
__device__ __forceinline__ bool inside_block(const BlockRec &b, const float p[3]) {
    return p[0] >= b.lo[0] && p[0] < b.hi[0] && p[1] >= b.lo[1] && p[1] < b.hi[1] && p[2] >= b.lo[2] &&
           p[2] <= b.hi[2];
}

// Continuous vertex coordinate along one axis: (p - lo) * k.
__device__ __forceinline__ float axis_coord(float p, float lo, float k) { return __fmul_rn(__fsub_rn(p, lo), k); }

// --- unbounded blocks: the region they own and the contraction (Eq. 16) -----
// The block owns its xy footprint extended to infinity across the sides in
// b.unb (half-open as Eq. 4) and every z.
__device__ __forceinline__ bool owned_unbounded(const BlockRec &b, const float p[3]) {
    const int e = b.unb;
    return ((e & kUnbXLo) || p[0] >= b.lo[0]) && ((e & kUnbXHi) || p[0] < b.hi[0]) &&
           ((e & kUnbYLo) || p[1] >= b.lo[1]) && ((e & kUnbYHi) || p[1] < b.hi[1]);
}

// x = (p - c) * (2 / (hi - lo)) and ||x||_inf, then u = contract(x): x inside
// the unit cube; outside, 2 - 1/|x_j| (sign of x_j) on the coordinates that
// reach the norm and x_j / ||x|| on the rest.  FP32, round to nearest.
__device__ __forceinline__ float unbounded_x(const BlockRec &b, const float p[3], float x[3]) {
    float m = 0.f;
#pragma unroll
    for (int a = 0; a < 3; a++) {
        x[a] = __fmul_rn(__fsub_rn(p[a], b.cc[a]), b.ih[a]);
        m = fmaxf(m, fabsf(x[a]));
    }
    return m;
}

__device__ __forceinline__ void contract_u(const float x[3], float m, float u[3]) {
#pragma unroll
    for (int a = 0; a < 3; a++) {
        if (m <= 1.f) {
            u[a] = x[a];
        } else if (fabsf(x[a]) == m) {
            const float v = __fsub_rn(2.f, __fdiv_rn(1.f, fabsf(x[a])));
            u[a] = x[a] < 0.f ? -v : v;
        } else {
            u[a] = __fdiv_rn(x[a], m);
        }
    }
}

// Lookup coordinates of a point for the feature gathers: q (the point, or
// its contraction u for an unbounded block) and the grid coordinate g.
__device__ __forceinline__ void lookup_coords(const BlockRec &b, const float p[3], float q[3], float g[3]) {
    if (b.unb & kUnbContracted) {
        float x[3];
        const float m = unbounded_x(b, p, x);
        contract_u(x, m, q);
    } else {
#pragma unroll
        for (int a = 0; a < 3; a++) q[a] = p[a];
    }
#pragma unroll
    for (int a = 0; a < 3; a++) g[a] = axis_coord(q[a], b.plo[a], b.kg[a]);
}

// Candidate lattice range of a ray in a block: FP32 slab test on the grown
// box, widened by two indices at each end.  Returns false on a miss.
__device__ __forceinline__ bool candidate_range(const BlockRec &b, const float o[3], const float d[3],
                                                const float inv_d[3], int &i0, int &i1, float &tfar) {
    float tn = 0.f, tf = 3.0e38f;
#pragma unroll
    for (int a = 0; a < 3; a++) {
        const float lo = b.lo_e[a], hi = b.hi_e[a];
        if (d[a] == 0.f) {
            if (o[a] < lo || o[a] > hi) return false;
        } else {
            const float inv = inv_d[a];
            const float t0 = (lo - o[a]) * inv, t1 = (hi - o[a]) * inv;
            tn = fmaxf(tn, fminf(t0, t1));
            tf = fminf(tf, fmaxf(t0, t1));
        }
    }
    if (!(tn <= tf)) return false;
    const float inv_delta = 1.0f / b.delta;
    const float a0 = floorf(tn * inv_delta - 0.5f) - 2.f;
    const float a1 = ceilf(tf * inv_delta - 0.5f) + 2.f;
    i0 = a0 < 0.f ? 0 : a0 > 2.0e9f ? 2000000000 : (int)a0;
    i1 = a1 > 2.0e9f ? 2000000000 : (int)a1;
    tfar = tf;
    return i1 >= i0;
}

// ---------------------------------------------------------------------------
// TMA bulk copy global -> shared with an mbarrier, and a bounded wait

__device__ __forceinline__ uint32_t smem_addr(const void *p) {
    return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ void mbar_init(uint64_t *bar, unsigned count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(bar)), "r"(count) : "memory");
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

// one elected thread: announce `bytes` and start the copy (16-byte aligned, multiple of 16)
__device__ __forceinline__ void bulk_copy_g2s(void *dst, const void *src, unsigned bytes, uint64_t *bar) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_addr(bar)), "r"(bytes)
                 : "memory");
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                     smem_addr(dst)),
                 "l"(src), "r"(bytes), "r"(smem_addr(bar))
                 : "memory");
}

// Wait for phase `parity` of the barrier, giving up after `limit` polls.
__device__ __forceinline__ bool mbar_wait(uint64_t *bar, unsigned parity, unsigned limit) {
    const uint32_t a = smem_addr(bar);
    for (unsigned it = 0; it < limit; it++) {
        uint32_t ok;
        asm volatile(
            "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}"
            : "=r"(ok)
            : "r"(a), "r"(parity)
            : "memory");
        if (ok) return true;
    }
    return false;
}

// ---------------------------------------------------------------------------
// storage loads: 8 channels of one vertex / texel as float (unscaled)

// L1 (and L2) cache policy of a read-only feature gather.
enum LdPolicy {
    kLdNormal = 0,
    kLdEvictFirst = 1,           // L1::evict_first
    kLdEvictLast = 2,            // L1::evict_last
    kLdNoAllocate = 3,           // L1::no_allocate
    kLdNoAllocateL2First = 4,    // L1::no_allocate, L2 evict_first
    kLdL2Last = 5,               // L2 evict_last
    kLdNoAllocateL2Last = 6,     // L1::no_allocate, L2 evict_last
};

#define COW_LD256(QUAL)                                                                                          \
    asm("ld.global.nc" QUAL ".v8.b32 {%0,%1,%2,%3,%4,%5,%6,%7}, [%8];"                                           \
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7])         \
        : "l"(p))

// 256-bit non-coherent global load (sm_100+); p must be 32-byte aligned.  The
// data is read-only for the kernel's lifetime, so the asm has no side effects
// and the compiler may schedule it freely.
#define COW_LD256_L2(QUAL, FRAC)                                                                                 \
    asm("{\n\t.reg .b64 pol;\n\tcreatepolicy.fractional." FRAC ".b64 pol, 1.0;\n\t"                              \
        "ld.global.nc" QUAL ".L2::cache_hint.v8.b32 {%0,%1,%2,%3,%4,%5,%6,%7}, [%8], pol;\n\t}"                      \
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7])         \
        : "l"(p))

template <int POL = kLdNormal>
__device__ __forceinline__ void ld256(const void *p, uint32_t r[8]) {
    if constexpr (POL == kLdEvictFirst) COW_LD256(".L1::evict_first");
    else if constexpr (POL == kLdEvictLast) COW_LD256(".L1::evict_last");
    else if constexpr (POL == kLdNoAllocate) COW_LD256(".L1::no_allocate");
    else if constexpr (POL == kLdNoAllocateL2First) COW_LD256_L2(".L1::no_allocate", "L2::evict_first");
    else if constexpr (POL == kLdL2Last) COW_LD256_L2("", "L2::evict_last");
    else if constexpr (POL == kLdNoAllocateL2Last) COW_LD256_L2(".L1::no_allocate", "L2::evict_last");
    else COW_LD256("");
}
#undef COW_LD256
#undef COW_LD256_L2

// 128-bit non-coherent global load with the same policies; p 16-byte aligned.
#define COW_LD128(QUAL) \
    asm("ld.global.nc" QUAL ".v4.b32 {%0,%1,%2,%3}, [%4];" : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]) : "l"(p))
#define COW_LD128_L2(QUAL, FRAC)                                                                                 \
    asm("{\n\t.reg .b64 pol;\n\tcreatepolicy.fractional." FRAC ".b64 pol, 1.0;\n\t"                              \
        "ld.global.nc" QUAL ".L2::cache_hint.v4.b32 {%0,%1,%2,%3}, [%4], pol;\n\t}"                                \
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3])                                                         \
        : "l"(p))

template <int POL = kLdNormal>
__device__ __forceinline__ void ld128(const void *p, uint32_t r[4]) {
    if constexpr (POL == kLdEvictFirst) COW_LD128(".L1::evict_first");
    else if constexpr (POL == kLdEvictLast) COW_LD128(".L1::evict_last");
    else if constexpr (POL == kLdNoAllocate) COW_LD128(".L1::no_allocate");
    else if constexpr (POL == kLdNoAllocateL2First) COW_LD128_L2(".L1::no_allocate", "L2::evict_first");
    else if constexpr (POL == kLdL2Last) COW_LD128_L2("", "L2::evict_last");
    else if constexpr (POL == kLdNoAllocateL2Last) COW_LD128_L2(".L1::no_allocate", "L2::evict_last");
    else COW_LD128("");
}
#undef COW_LD128
#undef COW_LD128_L2

__device__ __forceinline__ float2 bf16x2_to_float2(uint32_t w) {
    // a bfloat16 is the upper half of the float with the same value
    return make_float2(__uint_as_float(w << 16), __uint_as_float(w & 0xffff0000u));
}

__device__ __forceinline__ float2 f16x2_to_float2(uint32_t w) {
    return __half22float2(*reinterpret_cast<const __half2 *>(&w));
}

__device__ __forceinline__ float2 fp8x2_to_float2(uint32_t w16) {
    const __half2_raw hr = __nv_cvt_fp8x2_to_halfraw2((__nv_fp8x2_storage_t)(w16 & 0xffffu), __NV_E4M3);
    return __half22float2(*reinterpret_cast<const __half2 *>(&hr));
}

// Storage loaders.  FP32 keeps the natural layout: one 32-byte vertex per
// 256-bit load.  The 16- and 8-bit formats use the pair layout: element i
// holds vertex i and vertex i+1 of the same row (x for the grid, u for the
// planes; the last element of a row repeats its vertex), so one load returns
// both corners of an interpolation pair.  Channels come as four float2
// pairs (c0 c1 | c2 c3 | c4 c5 | c6 c7).
template <int DT>
struct Store;

template <>
struct Store<kF32> {
    static constexpr bool kPaired = false;
    template <int POL = kLdNormal>
    __device__ __forceinline__ static void load8(const void *base, int64_t idx, float2 v[4]) {
        uint32_t r[8];
        ld256<POL>(reinterpret_cast<const uint4 *>(base) + 2 * idx, r);
#pragma unroll
        for (int k = 0; k < 4; k++) v[k] = make_float2(__uint_as_float(r[2 * k]), __uint_as_float(r[2 * k + 1]));
    }
    template <int POL = kLdNormal>
    __device__ __forceinline__ static void load_pair(const void *, int64_t, float2[4], float2[4]) {}
};

template <>
struct Store<kF16> {
    static constexpr bool kPaired = true;
    template <int POL = kLdNormal>
    __device__ __forceinline__ static void load8(const void *, int64_t, float2[4]) {}
    template <int POL = kLdNormal>
    __device__ __forceinline__ static void load_pair(const void *base, int64_t idx, float2 lo[4], float2 hi[4]) {
        uint32_t r[8];
        ld256<POL>(reinterpret_cast<const uint4 *>(base) + 2 * idx, r);
#pragma unroll
        for (int k = 0; k < 4; k++) {
            lo[k] = f16x2_to_float2(r[k]);
            hi[k] = f16x2_to_float2(r[4 + k]);
        }
    }
};

template <>
struct Store<kBF16> {
    static constexpr bool kPaired = true;
    template <int POL = kLdNormal>
    __device__ __forceinline__ static void load8(const void *, int64_t, float2[4]) {}
    template <int POL = kLdNormal>
    __device__ __forceinline__ static void load_pair(const void *base, int64_t idx, float2 lo[4], float2 hi[4]) {
        uint32_t r[8];
        ld256<POL>(reinterpret_cast<const uint4 *>(base) + 2 * idx, r);
#pragma unroll
        for (int k = 0; k < 4; k++) {
            lo[k] = bf16x2_to_float2(r[k]);
            hi[k] = bf16x2_to_float2(r[4 + k]);
        }
    }
};

template <>
struct Store<kFP8> {
    static constexpr bool kPaired = true;
    template <int POL = kLdNormal>
    __device__ __forceinline__ static void load8(const void *, int64_t, float2[4]) {}
    template <int POL = kLdNormal>
    __device__ __forceinline__ static void load_pair(const void *base, int64_t idx, float2 lo[4], float2 hi[4]) {
        const uint4 q = __ldg(reinterpret_cast<const uint4 *>(base) + idx);
        lo[0] = fp8x2_to_float2(q.x);
        lo[1] = fp8x2_to_float2(q.x >> 16);
        lo[2] = fp8x2_to_float2(q.y);
        lo[3] = fp8x2_to_float2(q.y >> 16);
        hi[0] = fp8x2_to_float2(q.z);
        hi[1] = fp8x2_to_float2(q.z >> 16);
        hi[2] = fp8x2_to_float2(q.w);
        hi[3] = fp8x2_to_float2(q.w >> 16);
    }
};

// BF16 grid of the mixed format (its planes are read by accumulate_sample)
template <>
struct Store<kMixed> : Store<kBF16> {};

// kFP8D: its quad-layout grid and planes are read by accumulate_sample
template <>
struct Store<kFP8D> {
    static constexpr bool kPaired = false;
    template <int POL = kLdNormal>
    __device__ __forceinline__ static void load8(const void *, int64_t, float2[4]) {}
    template <int POL = kLdNormal>
    __device__ __forceinline__ static void load_pair(const void *, int64_t, float2[4], float2[4]) {}
};

__device__ __forceinline__ float sigmoidf_fast(float x) { return __fdividef(1.0f, 1.0f + __expf(-x)); }

// Host: calls f(std::integral_constant<int, DT>{}) with the kernel variant of
// a kernel dtype (storage, | kBrickBit for brick-sparse grids); returns its
// result, or cudaErrorInvalidValue for an unknown dtype.
template <class F>
inline cudaError_t dispatch_dt(int dt, F &&f) {
#define COW_DT_CASE(V) \
    case (V): return f(std::integral_constant<int, (V)>{});
    switch (dt) {
        COW_DT_CASE(kF32)
        COW_DT_CASE(kF16)
        COW_DT_CASE(kBF16)
        COW_DT_CASE(kFP8)
        COW_DT_CASE(kMixed)
        COW_DT_CASE(kFP8D)
        COW_DT_CASE(kF32 | kBrickBit)
        COW_DT_CASE(kF16 | kBrickBit)
        COW_DT_CASE(kBF16 | kBrickBit)
        COW_DT_CASE(kFP8 | kBrickBit)
        COW_DT_CASE(kMixed | kBrickBit)
        COW_DT_CASE(kFP8D | kBrickBit)
    default: return cudaErrorInvalidValue;
    }
#undef COW_DT_CASE
}

}  // namespace cow
