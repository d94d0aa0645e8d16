// march_core.cuh -- the sample sequence of a ray and the feature lookup, shared
// by the forward marcher and the backward pass so that both visit exactly the
// same samples.
#pragma once

#include "cow_common.cuh"

// Cache policies of the feature gathers, chosen by measurement on the 1080p
// LOD city: plane texels are rarely re-read from L1 by neighbouring rays
// (the planes are 4x finer than the grid), so they bypass L1 and leave it to
// the grid; grid lines are kept in L2 ahead of plane lines, while the planes
// still depend on L2 (an L2 evict-first hint on them halves the frame rate).
#ifndef COW_GRID_LD_POLICY
#define COW_GRID_LD_POLICY 5
#endif
#ifndef COW_PLANE_LD_POLICY
#define COW_PLANE_LD_POLICY 6
#endif

namespace cow {

// L1 policies of the grid and plane gathers (LdPolicy)
constexpr int kGridLd = COW_GRID_LD_POLICY;
constexpr int kPlaneLd = COW_PLANE_LD_POLICY;

// Feature lookup f^{k,l}(p): trilinear grid + bilinear xy, xz, yz planes.
// g: the FP32 grid coordinate the cell decision computed.  The 8 channels are
// accumulated as four float2 pairs with packed FP32 FMA (same rounding per
// element as scalar FMA).
//
// The grid element of the voxel's first corner is found directly (dense) or
// through the block's brick table (brick-sparse: the brick of the voxel, then
// the voxel's place inside it); the other corners are at the layout's fixed
// strides from it.  A voxel whose brick is not stored (only a lookup at an
// arbitrary point can meet one: lattice samples lie in occupied cells, whose
// bricks are stored) reads no grid element and takes the grid term as zero;
// callers that pass a BrickCache march lattice samples and skip that test.
// The brick slot of the last lookup of one ray in one block (brick-sparse
// grids): successive samples mostly stay in one 16^3-voxel brick, so the
// table read leaves the gathers' address path.
struct BrickCache {
    int key = -1;
    int slot = 0;
};

template <int DT>
__device__ __forceinline__ void accumulate_sample(const BlockRec &b, const float p[3], const float g[3], float2 f[4],
                                                  BrickCache *bc = nullptr) {
    constexpr int ST = DT & kStoreMask;                 // storage format
    constexpr bool kBricks = (DT & kBrickBit) != 0;     // brick-sparse grid
    float fr[3];
    int c0[3];
#pragma unroll
    for (int a = 0; a < 3; a++) {
        const int v = min(max(__float2int_rd(g[a]), 0), b.R - 2);
        c0[a] = v;
        fr[a] = fminf(fmaxf(g[a], 0.f), (float)(b.R - 1)) - (float)v;
    }
    const int R = b.R;
    int64_t base, dbase = 0;
    int sy, sz;
    bool stored = true;
    if constexpr (kBricks) {
        const int nb = b.Nb;
        const int key = ((c0[2] >> kBrickLog2) * nb + (c0[1] >> kBrickLog2)) * nb + (c0[0] >> kBrickLog2);
        int slot;
        if (bc) {
            if (key != bc->key) {
                bc->key = key;
                bc->slot = __ldg(b.brick + key);
            }
            slot = bc->slot;
        } else {
            slot = __ldg(b.brick + key);
        }
        sy = b.bsy;
        sz = b.bsz;
        const int loc = (c0[2] & (kBrick - 1)) * sz + (c0[1] & (kBrick - 1)) * sy + (c0[0] & (kBrick - 1));
        base = (int64_t)slot * b.belem + loc;
        dbase = (int64_t)slot * kDensBrickElems + loc;
        // a lattice sample (the callers that pass a cache) lies in an
        // occupied cell, whose brick is stored; only a lookup at an
        // arbitrary point can meet an empty brick
        stored = bc != nullptr || slot >= 0;
    } else {
        base = ((int64_t)c0[2] * R + c0[1]) * R + c0[0];
        dbase = base;
        sy = R;
        sz = R * R;
    }
    float2 acc[4];
#pragma unroll
    for (int c = 0; c < 4; c++) acc[c] = make_float2(0.f, 0.f);
    const float wx[2] = {1.f - fr[0], fr[0]}, wy[2] = {1.f - fr[1], fr[1]}, wz[2] = {1.f - fr[2], fr[2]};
    float dens = 0.f;  // kFP8D: the BF16 log-density
    if (stored) {
        if constexpr (ST == kFP8D) {
            // the eight FP8 channels of slices z and z+1: one 32-byte quad each
#pragma unroll
            for (int dz = 0; dz < 2; dz++) {
                uint32_t r[8];
                ld256<kGridLd>(reinterpret_cast<const uint4 *>(b.grid) + 2 * (base + (int64_t)dz * sz), r);
#pragma unroll
                for (int q = 0; q < 4; q++) {
                    const float w = (wy[q >> 1] * wz[dz]) * wx[q & 1];
                    const float2 w2 = make_float2(w, w);
                    acc[0] = __ffma2_rn(w2, fp8x2_to_float2(r[2 * q]), acc[0]);
                    acc[1] = __ffma2_rn(w2, fp8x2_to_float2(r[2 * q] >> 16), acc[1]);
                    acc[2] = __ffma2_rn(w2, fp8x2_to_float2(r[2 * q + 1]), acc[2]);
                    acc[3] = __ffma2_rn(w2, fp8x2_to_float2(r[2 * q + 1] >> 16), acc[3]);
                }
            }
            // channel 0 from the BF16 octet: corners 2j and 2j+1 in word j
            uint32_t dv[4];
            ld128<kGridLd>(reinterpret_cast<const uint4 *>(b.dens) + dbase, dv);
#pragma unroll
            for (int j = 0; j < 4; j++) {
                const float2 v = bf16x2_to_float2(dv[j]);
                const float wyz = wy[j & 1] * wz[j >> 1];
                dens = fmaf(wyz * wx[1], v.y, fmaf(wyz * wx[0], v.x, dens));
            }
        } else if (Store<ST>::kPaired) {
            // four loads, each the x-pair of one (y, z) edge of the voxel
#pragma unroll
            for (int k = 0; k < 4; k++) {
                const int dy = k & 1, dz = k >> 1;
                const float wyz = wy[dy] * wz[dz];
                const float2 w0 = make_float2(wyz * wx[0], wyz * wx[0]), w1 = make_float2(wyz * wx[1], wyz * wx[1]);
                float2 lo[4], hi[4];
                const int64_t e = kBricks ? base + (int64_t)(dz * sz + dy * sy) : base + ((int64_t)dz * R + dy) * R;
                Store<ST>::template load_pair<kGridLd>(b.grid, e, lo, hi);
#pragma unroll
                for (int c = 0; c < 4; c++) acc[c] = __ffma2_rn(w1, hi[c], __ffma2_rn(w0, lo[c], acc[c]));
            }
        } else {
#pragma unroll
            for (int k = 0; k < 8; k++) {
                const int dx = k & 1, dy = (k >> 1) & 1, dz = k >> 2;
                const float w = (wy[dy] * wz[dz]) * wx[dx];
                const float2 w2 = make_float2(w, w);
                float2 v[4];
                const int64_t e =
                    kBricks ? base + (int64_t)(dz * sz + dy * sy + dx) : base + ((int64_t)dz * R + dy) * R + dx;
                Store<ST>::template load8<kGridLd>(b.grid, e, v);
#pragma unroll
                for (int c = 0; c < 4; c++) acc[c] = __ffma2_rn(w2, v[c], acc[c]);
            }
        }
    }
    // per-channel scales: 8 floats of one tensor as two 16-byte loads (the
    // scale array is its own allocation, so 16-byte aligned).  Plain loads:
    // the non-coherent path measured 4 % slower in the batched kernel, whose
    // records sit in shared memory, and equal in the view kernel.
    const float4 *scale4 = reinterpret_cast<const float4 *>(b.scale);
    if (ST == kFP8 || ST == kFP8D) {
        const float4 sa = scale4[0], sb = scale4[1];
        f[0] = make_float2(ST == kFP8D ? dens : acc[0].x * sa.x, acc[0].y * sa.y);
        f[1] = make_float2(acc[1].x * sa.z, acc[1].y * sa.w);
        f[2] = make_float2(acc[2].x * sb.x, acc[2].y * sb.y);
        f[3] = make_float2(acc[3].x * sb.z, acc[3].y * sb.w);
    } else {
#pragma unroll
        for (int c = 0; c < 4; c++) f[c] = acc[c];
    }
    // planes: vertex-aligned bilinear in (x, y), (x, z), (y, z)
    float hf[3];
    int h0[3];
#pragma unroll
    for (int a = 0; a < 3; a++) {
        float h = axis_coord(p[a], b.plo[a], b.kp[a]);
        const int u = min(max(__float2int_rd(h), 0), b.P - 2);
        h = fminf(fmaxf(h, 0.f), (float)(b.P - 1));
        h0[a] = u;
        hf[a] = h - (float)u;
    }
    const int P = b.P;
#pragma unroll
    for (int pl = 0; pl < 3; pl++) {
        const int ua = pl == 2 ? 1 : 0, va = pl == 0 ? 1 : 2;
        const int64_t tb = (int64_t)h0[va] * P + h0[ua];
        const float wu[2] = {1.f - hf[ua], hf[ua]}, wv[2] = {1.f - hf[va], hf[va]};
        float2 pacc[4];
#pragma unroll
        for (int c = 0; c < 4; c++) pacc[c] = make_float2(0.f, 0.f);
        if (ST == kMixed || ST == kFP8D) {
            // one 32-byte load: the 2x2 FP8 texels of the bilinear footprint
            // (hardware E4M3 conversions; an integer re-biasing of the bytes
            // measured 20 % slower)
            uint32_t r[8];
            ld256<kPlaneLd>(reinterpret_cast<const uint4 *>(b.planes[pl]) + 2 * tb, r);
#pragma unroll
            for (int q = 0; q < 4; q++) {
                const float w = wv[q >> 1] * wu[q & 1];
                const float2 w2 = make_float2(w, w);
                pacc[0] = __ffma2_rn(w2, fp8x2_to_float2(r[2 * q]), pacc[0]);
                pacc[1] = __ffma2_rn(w2, fp8x2_to_float2(r[2 * q] >> 16), pacc[1]);
                pacc[2] = __ffma2_rn(w2, fp8x2_to_float2(r[2 * q + 1]), pacc[2]);
                pacc[3] = __ffma2_rn(w2, fp8x2_to_float2(r[2 * q + 1] >> 16), pacc[3]);
            }
        } else if (Store<ST>::kPaired) {
#pragma unroll
            for (int dv = 0; dv < 2; dv++) {
                const float2 w0 = make_float2(wv[dv] * wu[0], wv[dv] * wu[0]);
                const float2 w1 = make_float2(wv[dv] * wu[1], wv[dv] * wu[1]);
                float2 lo[4], hi[4];
                Store<ST>::template load_pair<kPlaneLd>(b.planes[pl], tb + (int64_t)dv * P, lo, hi);
#pragma unroll
                for (int c = 0; c < 4; c++) pacc[c] = __ffma2_rn(w1, hi[c], __ffma2_rn(w0, lo[c], pacc[c]));
            }
        } else {
#pragma unroll
            for (int q = 0; q < 4; q++) {
                const int du = q & 1, dv = q >> 1;
                const float w = wv[dv] * wu[du];
                const float2 w2 = make_float2(w, w);
                float2 v[4];
                Store<ST>::template load8<kPlaneLd>(b.planes[pl], tb + (int64_t)dv * P + du, v);
#pragma unroll
                for (int c = 0; c < 4; c++) pacc[c] = __ffma2_rn(w2, v[c], pacc[c]);
            }
        }
        if (ST == kFP8 || ST == kMixed || ST == kFP8D) {
            const float4 sa = scale4[2 * (pl + 1)], sb = scale4[2 * (pl + 1) + 1];
            f[0] = __ffma2_rn(pacc[0], make_float2(sa.x, sa.y), f[0]);
            f[1] = __ffma2_rn(pacc[1], make_float2(sa.z, sa.w), f[1]);
            f[2] = __ffma2_rn(pacc[2], make_float2(sb.x, sb.y), f[2]);
            f[3] = __ffma2_rn(pacc[3], make_float2(sb.z, sb.w), f[3]);
        } else {
#pragma unroll
            for (int c = 0; c < 4; c++) f[c] = __fadd2_rn(f[c], pacc[c]);
        }
    }
}

// Visit the occupied lattice samples of one ray inside one block, in order
// (Eq. 4 membership, occupancy skip); fn(p, g, s) is called for each with
// the lookup point, the grid coordinate and the sample's step s (delta of
// Eq. 1), and returns false to stop the ray.  Returns false when fn stopped
// it.
//
// Two-level occupancy (Sec. 4.1's multi-level occupancy grid): a sample
// tests its own cell; when that is empty it tests the coarse cell around it
// (kOccGroup^3 cells, the OR of their bits) and leaves the larger of the two
// empty cells.  Empty cells are left with an exact jump: along each
// axis the FP32 cell index of successive lattice points is monotone (every
// step of the decision sequence is monotone, and so is the coarse index
// cell >> kOccGroupLog2), so every lattice point before the ray's exit from
// the empty cell -- shrunk by a margin m far above the FP32 position and
// coordinate error -- decides an empty cell and would be skipped anyway.
// The jump lands one lattice step short of that exit.
// First lattice index of the ray inside an unbounded block's region, or -1.
// The owned indices form one interval (convex region, monotone FP32 lattice
// coordinates); its start is found from the FP32 entry estimate
// j = floor(t_in / delta - 1/2) over the bounded xy sides by stepping back
// while the previous point is owned, or forward (at most 64 points) until one
// is.  The same FP32 sequence as the oracle's, so both find the same index.
__device__ __forceinline__ int first_owned_index(const BlockRec &b, const float o[3], const float d[3]) {
    float tn = 0.f;
#pragma unroll
    for (int a = 0; a < 2; a++) {
        const bool elo = b.unb & (a == 0 ? kUnbXLo : kUnbYLo), ehi = b.unb & (a == 0 ? kUnbXHi : kUnbYHi);
        if (d[a] == 0.f) {
            if ((!elo && o[a] < b.lo[a]) || (!ehi && o[a] >= b.hi[a])) return -1;
            continue;
        }
        if (d[a] > 0.f ? elo : ehi) continue;
        const float inv = __fdiv_rn(1.f, d[a]);
        const float bound = d[a] > 0.f ? b.lo[a] : b.hi[a];
        tn = fmaxf(tn, __fmul_rn(__fsub_rn(bound, o[a]), inv));
    }
    const float xs = __fsub_rn(__fmul_rn(tn, __fdiv_rn(1.f, b.delta)), 0.5f);
    if (!(xs < 16777216.f)) return -1;
    int j = max(__float2int_rd(xs), 0);
    float p[3];
    lattice_point(o, d, b.delta, j, p);
    if (owned_unbounded(b, p)) {
        for (int k = 0; k < 64 && j > 0; k++) {
            lattice_point(o, d, b.delta, j - 1, p);
            if (!owned_unbounded(b, p)) break;
            j--;
        }
        return j;
    }
    for (int k = 1; k <= 64; k++) {
        lattice_point(o, d, b.delta, j + k, p);
        if (owned_unbounded(b, p)) return j + k;
    }
    return -1;
}

// Samples of an unbounded (contracted) block: from its first owned lattice
// point the ray advances by s = (delta m) m, m = max(1, ||x||_inf) -- one
// lattice step inside the box, one lattice step of the dominant contracted
// coordinate outside -- until it leaves the region, ||x|| exceeds 1e4 or
// 65536 steps were taken.  Each occupied point calls fn(u, g, s).
template <typename Fn>
__device__ __forceinline__ bool for_each_sample_unbounded(const BlockRec &b, const float o[3], const float d[3],
                                                          Fn &&fn) {
    const int i0 = first_owned_index(b, o, d);
    if (i0 < 0) return true;
    const int Nc = b.Nc, C = b.C, R = b.R;
    float t = __fmul_rn(__fadd_rn(__int2float_rn(i0), 0.5f), b.delta);
    int occ_w = -1;
    uint32_t occ_bits = 0u;
    for (int k = 0; k < kContractSteps; k++) {
        float p[3];
#pragma unroll
        for (int a = 0; a < 3; a++) p[a] = __fadd_rn(o[a], __fmul_rn(t, d[a]));
        if (!owned_unbounded(b, p)) break;
        float x[3];
        const float m = unbounded_x(b, p, x);
        if (m > kContractMax) break;
        const float m1 = fmaxf(m, 1.f);
        const float s = __fmul_rn(__fmul_rn(b.delta, m1), m1);
        float u[3], g[3];
        contract_u(x, m, u);
        int cell[3];
#pragma unroll
        for (int a = 0; a < 3; a++) {
            g[a] = axis_coord(u[a], b.plo[a], b.kg[a]);
            const int v = min(max(__float2int_rd(g[a]), 0), R - 2);
            cell[a] = C == 1 ? v : (int)__umulhi((unsigned)v, b.cdiv);
        }
        const int ci = (cell[2] * Nc + cell[1]) * Nc + cell[0];
        if ((ci >> 5) != occ_w) {
            occ_w = ci >> 5;
            occ_bits = __ldg(b.occ + occ_w);
        }
        if ((occ_bits >> (ci & 31)) & 1u)
            if (!fn(u, g, s)) return false;
        t = __fadd_rn(t, s);
    }
    return true;
}

template <typename Fn>
__device__ __forceinline__ bool for_each_sample(const BlockRec &b, const float o[3], const float d[3],
                                                const float inv_d[3], float omax, unsigned *err, Fn &&fn) {
    if (b.unb & kUnbContracted) return for_each_sample_unbounded(b, o, d, fn);
    int i0, i1;
    float tfar;
    if (!candidate_range(b, o, d, inv_d, i0, i1, tfar)) return true;
    if (i1 - i0 > kMaxSpan) {
        atomicOr(err, kErrRange);
        i1 = i0 + kMaxSpan;
    }
    const float delta = b.delta, inv_delta = 1.0f / b.delta;
    const float m = 4e-6f * (omax + tfar + b.bmax);
    const int Nc = b.Nc, C = b.C, R = b.R, Nc2 = b.Nc2;
    // the occupancy words of the last lookups: a ray stays in one cell for
    // many lattice steps, so most lookups reuse them instead of a gather
    int occ_w = -1, occ2_w = -1;
    uint32_t occ_bits = 0u, occ2_bits = 0u;
    for (int i = i0; i <= i1; i++) {
        float p[3];
        lattice_point(o, d, delta, i, p);
        if (!inside_block(b, p)) continue;
        int cell[3];
        float g[3];
#pragma unroll
        for (int a = 0; a < 3; a++) {
            g[a] = axis_coord(p[a], b.lo[a], b.kg[a]);
            const int v = min(max(__float2int_rd(g[a]), 0), R - 2);
            cell[a] = C == 1 ? v : (int)__umulhi((unsigned)v, b.cdiv);
        }
        const int ci = (cell[2] * Nc + cell[1]) * Nc + cell[0];
        if ((ci >> 5) != occ_w) {
            occ_w = ci >> 5;
            occ_bits = __ldg(b.occ + occ_w);
        }
        if (!((occ_bits >> (ci & 31)) & 1u)) {
            // an empty cell; when its whole coarse cell is empty, leave that instead
            const int ci2 = ((cell[2] >> kOccGroupLog2) * Nc2 + (cell[1] >> kOccGroupLog2)) * Nc2 +
                            (cell[0] >> kOccGroupLog2);
            if ((ci2 >> 5) != occ2_w) {
                occ2_w = ci2 >> 5;
                occ2_bits = __ldg(b.occ2 + occ2_w);
            }
            const int lvl = ((occ2_bits >> (ci2 & 31)) & 1u) ? 0 : kOccGroupLog2;  // log2 cells per edge
            // exit of the empty cell: cells of C << lvl voxels, the last one
            // reaching the block's far face
            const int Ce = C << lvl, last = lvl ? Nc2 - 1 : Nc - 1;
            float tx = 3.0e38f;
#pragma unroll
            for (int a = 0; a < 3; a++) {
                const int ce = cell[a] >> lvl;
                if (d[a] > 0.f) {
                    const float chi = ce == last ? b.hi[a] : fmaf((float)((ce + 1) * Ce), b.vox[a], b.lo[a]);
                    tx = fminf(tx, (chi - m - o[a]) * inv_d[a]);
                } else if (d[a] < 0.f) {
                    const float clo = fmaf((float)(ce * Ce), b.vox[a], b.lo[a]);
                    tx = fminf(tx, (clo + m - o[a]) * inv_d[a]);
                }
            }
            const int j = __float2int_rd(tx * inv_delta - 0.5f) - 1;
            if (j > i) i = min(j, i1);
            continue;
        }
        if (!fn(p, g, delta)) return false;
    }
    return true;
}

__device__ __forceinline__ void ray_setup(const float d[3], const float o[3], float inv_d[3], float &omax) {
#pragma unroll
    for (int a = 0; a < 3; a++) inv_d[a] = d[a] != 0.f ? 1.0f / d[a] : 0.f;
    omax = fmaxf(fabsf(o[0]), fmaxf(fabsf(o[1]), fabsf(o[2])));
}

// Per-ray depth order of the ray-batch form: xy distance of block centres to
// this ray's origin (App. D) as the FP32 key dx*dx + dy*dy, ties by id.
// order[] receives positions into rr (block rr.id[k] is record rr.r[k]).
__device__ __forceinline__ int sort_blocks_for_ray(const RayRecs &rr, const float o[3], int order[kMaxRayIds]) {
    float key[kMaxRayIds];
    const int n = rr.n;
    for (int i = 0; i < n; i++) {
        const BlockRec &b = rr.r[i];
        const int id = rr.id[i];
        const float dx = __fsub_rn(b.cx, o[0]), dy = __fsub_rn(b.cy, o[1]);
        const float kk = __fadd_rn(__fmul_rn(dx, dx), __fmul_rn(dy, dy));
        int j = i - 1;
        while (j >= 0 && (key[j] > kk || (key[j] == kk && rr.id[order[j]] > id))) {
            key[j + 1] = key[j];
            order[j + 1] = order[j];
            j--;
        }
        key[j + 1] = kk;
        order[j + 1] = i;
    }
    return n;
}

// Per-ray compositing state: C_d, F, the transmittance, occupied samples.
struct RayState {
    float Cd[3], F[4], T;
    int nsamp;
    bool done;
};

// March one ray through one block, updating its state (Eq. 1-2); when tb
// is given it is multiplied by every sample's 1 - alpha (the block's own
// transmittance, Eq. 11).
template <int DT>
__device__ __forceinline__ void march_block(const BlockRec &b, const float o[3], const float d[3],
                                            const float inv_d[3], float omax, float ert_eps, RayState &s,
                                            unsigned *err, float *tb = nullptr) {
    BrickCache bc;
    const bool more = for_each_sample(b, o, d, inv_d, omax, err, [&](const float p[3], const float g[3], float dt) {
        float2 f2[4];
        accumulate_sample<DT>(b, p, g, f2, &bc);
        const float f[8] = {f2[0].x, f2[0].y, f2[1].x, f2[1].y, f2[2].x, f2[2].y, f2[3].x, f2[3].y};
        const float sigma = __expf(f[0]);
        const float e = __expf(-sigma * dt);
        const float w = s.T * (1.f - e);
#pragma unroll
        for (int c = 0; c < 3; c++) s.Cd[c] = fmaf(w, sigmoidf_fast(f[1 + c]), s.Cd[c]);
#pragma unroll
        for (int c = 0; c < 4; c++) s.F[c] = fmaf(w, sigmoidf_fast(f[4 + c]), s.F[c]);
        s.T *= e;
        if (tb) *tb *= e;
        s.nsamp++;
        return !(s.T < ert_eps);
    });
    if (!more) s.done = true;
}

__device__ __forceinline__ float bf16r(float x) { return __bfloat162float(__float2bfloat16_rn(x)); }

// Deferred MLP (Eq. 3) from weights in shared memory.
__device__ __forceinline__ void deferred_mlp(const float *w, const float x_in[10], bool bf16, float out[3]) {
    float x[10];
#pragma unroll
    for (int i = 0; i < 10; i++) x[i] = bf16 ? bf16r(x_in[i]) : x_in[i];
    float h1[16];
#pragma unroll
    for (int j = 0; j < 16; j++) {
        float a = w[kOffB1 + j];
#pragma unroll
        for (int i = 0; i < 10; i++) a = fmaf(x[i], w[kOffW1 + i * 16 + j], a);
        a = fmaxf(a, 0.f);
        h1[j] = bf16 ? bf16r(a) : a;
    }
    float h2[16];
#pragma unroll
    for (int j = 0; j < 16; j++) {
        float a = w[kOffB2 + j];
#pragma unroll
        for (int i = 0; i < 16; i++) a = fmaf(h1[i], w[kOffW2 + i * 16 + j], a);
        a = fmaxf(a, 0.f);
        h2[j] = bf16 ? bf16r(a) : a;
    }
#pragma unroll
    for (int j = 0; j < 3; j++) {
        float a = w[kOffB3 + j];
#pragma unroll
        for (int i = 0; i < 16; i++) a = fmaf(h2[i], w[kOffW3 + i * 3 + j], a);
        out[j] = sigmoidf_fast(a);
    }
}

// Per-block deferred MLP Phi^k (Eq. 3 with block k's weights, read from
// global memory: the weight addresses are the same for every lane of a warp,
// so each load is one broadcast).  Input [C_d^k, F^k, PE(d)], PE(d) = d, then
// sin(2^l d) and cos(2^l d) for l < n_freq; weights input-major with
// n_in = 10 + 6 n_freq rows in W1.
__device__ __forceinline__ void mlp_row16(const float *__restrict__ row, float x, float h[16]) {
    const float4 *r4 = reinterpret_cast<const float4 *>(row);
#pragma unroll
    for (int q = 0; q < 4; q++) {
        const float4 r = __ldg(r4 + q);
        h[4 * q + 0] = fmaf(x, r.x, h[4 * q + 0]);
        h[4 * q + 1] = fmaf(x, r.y, h[4 * q + 1]);
        h[4 * q + 2] = fmaf(x, r.z, h[4 * q + 2]);
        h[4 * q + 3] = fmaf(x, r.w, h[4 * q + 3]);
    }
}

__device__ __forceinline__ void block_mlp(const float *__restrict__ w, int n_freq, const float cd[3], const float f[4],
                                          const float d[3], float out[3]) {
    const int n_in = 10 + 6 * n_freq;
    const float *b1 = w + n_in * 16, *W2 = b1 + 16, *b2 = W2 + 256, *W3 = b2 + 16, *b3 = W3 + 48;
    float h[16];
#pragma unroll
    for (int j = 0; j < 16; j++) h[j] = __ldg(b1 + j);
#pragma unroll
    for (int i = 0; i < 3; i++) mlp_row16(w + i * 16, cd[i], h);
#pragma unroll
    for (int i = 0; i < 4; i++) mlp_row16(w + (3 + i) * 16, f[i], h);
#pragma unroll
    for (int i = 0; i < 3; i++) mlp_row16(w + (7 + i) * 16, d[i], h);
    float sc = 1.0f;  // 2^l
#pragma unroll 1
    for (int l = 0; l < n_freq; l++) {
        const float *rows = w + (10 + 6 * l) * 16;
#pragma unroll
        for (int a = 0; a < 3; a++) {
            float sn, cs;
            sincosf(sc * d[a], &sn, &cs);
            mlp_row16(rows + a * 16, sn, h);
            mlp_row16(rows + (3 + a) * 16, cs, h);
        }
        sc *= 2.0f;
    }
#pragma unroll
    for (int j = 0; j < 16; j++) h[j] = fmaxf(h[j], 0.f);
    float h2[16];
#pragma unroll
    for (int j = 0; j < 16; j++) h2[j] = __ldg(b2 + j);
#pragma unroll
    for (int i = 0; i < 16; i++) mlp_row16(W2 + i * 16, h[i], h2);
#pragma unroll
    for (int j = 0; j < 3; j++) {
        float a = __ldg(b3 + j);
#pragma unroll
        for (int i = 0; i < 16; i++) a = fmaf(fmaxf(h2[i], 0.f), __ldg(W3 + i * 3 + j), a);
        out[j] = sigmoidf_fast(a);
    }
}

__device__ __forceinline__ void load_mlp(const float *g, float *s, bool bf16) {
    for (int i = threadIdx.x; i < kMlpParams; i += blockDim.x) {
        const float v = __ldg(g + i);
        // biases stay FP32 (they add into the FP32 accumulator)
        const bool is_bias = (i >= kOffB1 && i < kOffW2) || (i >= kOffB2 && i < kOffW3) || i >= kOffB3;
        s[i] = (bf16 && !is_bias) ? bf16r(v) : v;
    }
}

}  // namespace cow
