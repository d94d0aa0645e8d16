// march_kernels.cuh -- K1 ray marcher with in-register block compositor and the fused
// K3 deferred-MLP epilogue.
//
// Per pixel (Sec. 4.2 rendering stage):
//   for each selected block, near to far (App. D depth sort):
//     for each lattice sample of the ray inside the block (Eq. 4 membership)
//       skip it when its occupancy cell is empty (Sec. 4.1, Sec. 4.5)
//       f = trilinear(grid) + bilinear(xy) + bilinear(xz) + bilinear(yz)
//       sigma = exp(f0), alpha = 1 - exp(-sigma delta)            (Eq. 1)
//       C_d += T alpha sigmoid(f1..3), F += T alpha sigmoid(f4..7) (Eq. 2)
//       T *= 1 - alpha
//   Carrying T across blocks is Eq. 12 with Eq. 13 (1 - alpha^k equals the
//   product of the block's (1 - alpha_i)), so no per-block partials exist.
//   C = C_d + sigmoid(MLP(C_d, F, d))                                (Eq. 3)
#pragma once

#include "cow_common.cuh"
#include "cow_kernels.h"
#include "kernel_launch.h"
#include "march_core.cuh"

#ifndef COW_MARCH_MIN_BLOCKS
#define COW_MARCH_MIN_BLOCKS 4
#endif
#ifndef COW_MARCH_MIN_BLOCKS_W
#define COW_MARCH_MIN_BLOCKS_W 4
#endif
#ifndef COW_RAYS_MIN_BLOCKS
#define COW_RAYS_MIN_BLOCKS COW_MARCH_MIN_BLOCKS  // 2 or 3 measured slower on the 2x2-block fit
#endif
#ifndef COW_WARP_W
#define COW_WARP_W 8  // pixels per warp row (the warp covers COW_WARP_W x 32/COW_WARP_W pixels)
#endif

namespace cow {

namespace {

constexpr int kTileW = 16, kTileH = 8, kThreads = 128;
constexpr int kWarpW = COW_WARP_W, kWarpH = 32 / kWarpW;  // one ray per thread: a warp's pixel patch
static_assert(kTileW % kWarpW == 0 && kTileH % kWarpH == 0 && (kTileW / kWarpW) * (kTileH / kWarpH) == kThreads / 32,
              "the CTA tile is an exact grid of warp patches");
constexpr int kMinBlocks = COW_MARCH_MIN_BLOCKS;  // CTAs per SM the register budget is sized for
constexpr int kMinBlocksW = COW_MARCH_MIN_BLOCKS_W;
constexpr int kMaxSmemRecs = 96;                  // block records a CTA stages in shared memory
constexpr unsigned kWaitPolls = 1u << 24;         // bound on mbarrier polls



__device__ __forceinline__ void write_outputs(const MarchArgs &a, int64_t row, const RayState &s, const float d[3],
                                              const float *w_mlp) {
    float x[10] = {s.Cd[0], s.Cd[1], s.Cd[2], s.F[0], s.F[1], s.F[2], s.F[3], d[0], d[1], d[2]};
    float o[3];
    deferred_mlp(w_mlp, x, (a.flags & 1u) != 0, o);
    float *rgb = a.out_rgb + 3 * row;
    rgb[0] = s.Cd[0] + o[0];
    rgb[1] = s.Cd[1] + o[1];
    rgb[2] = s.Cd[2] + o[2];
    if (a.out_aux) {
        float4 *ap = reinterpret_cast<float4 *>(a.out_aux + 8 * row);
        ap[0] = make_float4(s.Cd[0], s.Cd[1], s.Cd[2], s.F[0]);
        ap[1] = make_float4(s.F[1], s.F[2], s.F[3], s.T);
    }
    if (a.out_nsamp) a.out_nsamp[row] = s.nsamp;
}

// View of a tile: views are ordered by tile_begin.
__device__ __forceinline__ int view_of_tile(const MarchArgs &a, int tile) {
    int lo = 0, hi = a.n_views - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (a.views[mid].tile_begin <= tile) lo = mid;
        else hi = mid - 1;
    }
    return lo;
}

// Per-block MLP form (Eq. 5 with Eq. 3 per block): every block is marched
// from an in-block transmittance of 1 (its C_d^k, F^k and 1 - alpha^k, Eq. 1-2
// / Eq. 11), a block with occupied samples adds T C^k with its own MLP, and
// T carries the product of the blocks' 1 - alpha^k.  Early termination uses
// the ray's total transmittance: inside block k it stops once
// T_k < ert_eps / T.  rec_at(k) / mlp_at(k): the k-th block's record and
// MLP weights in near-to-far order.
// state(k): where the k-th block's state goes (a.out_block_state, ray mode),
// or null.
template <int DT, class RecAt, class MlpAt, class StateAt>
__device__ __forceinline__ void blend_blocks(const MarchArgs &a, int n_blk, RecAt rec_at, MlpAt mlp_at,
                                             StateAt state, const float o[3], const float d[3],
                                             const float inv_d[3], float omax, int64_t row) {
    float C[3] = {0.f, 0.f, 0.f}, Cd[3] = {0.f, 0.f, 0.f}, F[4] = {0.f, 0.f, 0.f, 0.f}, T = 1.f;
    int nsamp = 0;
    for (int k = 0; k < n_blk; k++) {
        RayState sb = {{0.f, 0.f, 0.f}, {0.f, 0.f, 0.f, 0.f}, 1.f, 0, false};
        march_block<DT>(rec_at(k), o, d, inv_d, omax, a.ert_eps > 0.f ? a.ert_eps / T : 0.f, sb, a.err);
        if (float *e = state(k)) {
            float4 *e4 = reinterpret_cast<float4 *>(e);
            if (sb.nsamp == 0) {
                e4[0] = make_float4(0.f, 0.f, 0.f, 0.f);
                e4[1] = make_float4(0.f, 0.f, 0.f, -1.f);
            } else {
                e4[0] = make_float4(sb.Cd[0], sb.Cd[1], sb.Cd[2], sb.F[0]);
                e4[1] = make_float4(sb.F[1], sb.F[2], sb.F[3], T);
            }
        }
        if (sb.nsamp == 0) continue;
        float phi[3];
        block_mlp(mlp_at(k), a.n_freq, sb.Cd, sb.F, d, phi);
#pragma unroll
        for (int c = 0; c < 3; c++) {
            C[c] = fmaf(T, sb.Cd[c] + phi[c], C[c]);
            Cd[c] = fmaf(T, sb.Cd[c], Cd[c]);
        }
#pragma unroll
        for (int c = 0; c < 4; c++) F[c] = fmaf(T, sb.F[c], F[c]);
        T *= sb.T;
        nsamp += sb.nsamp;
        if (sb.done) break;
    }
    float *rgb = a.out_rgb + 3 * row;
    rgb[0] = C[0];
    rgb[1] = C[1];
    rgb[2] = C[2];
    if (a.out_aux) {
        float4 *ap = reinterpret_cast<float4 *>(a.out_aux + 8 * row);
        ap[0] = make_float4(Cd[0], Cd[1], Cd[2], F[0]);
        ap[1] = make_float4(F[1], F[2], F[3], T);
    }
    if (a.out_nsamp) a.out_nsamp[row] = nsamp;
}

template <int DT>
__device__ __forceinline__ void march_blocks_blend(const MarchArgs &a, const ViewRec &v, const BlockRec *recs,
                                                   const float o[3], const float d[3], const float inv_d[3],
                                                   float omax, int64_t row) {
    blend_blocks<DT>(
        a, v.ids_count, [&](int k) -> const BlockRec & { return recs[k]; },
        [&](int k) { return a.block_mlps[v.ids_begin + k]; }, [](int) -> float * { return nullptr; }, o, d, inv_d,
        omax, row);
}

// One ray per thread of the tile: march the view's near-to-far block list
// recs[0 .. ids_count) and write the pixel.
template <int DT, bool kBlockMlp>
__device__ __forceinline__ void march_tile_rays(const MarchArgs &a, const ViewRec &v, const BlockRec *recs, int tile,
                                                const float *s_mlp) {
    const int t = tile - v.tile_begin;
    int tx, ty;
    tile_xy(v, t, kTileH, tx, ty);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    constexpr int kWarpsX = kTileW / kWarpW;
    const int px = tx * kTileW + (warp % kWarpsX) * kWarpW + (lane % kWarpW);
    const int py = ty * kTileH + (warp / kWarpsX) * kWarpH + (lane / kWarpW);
    if (px >= v.W || py >= v.H) return;
    float o[3], d[3], inv_d[3], omax;
    pixel_ray(v, px, py, o, d);
    ray_setup(d, o, inv_d, omax);
    const int64_t row = v.pix_offset + (int64_t)py * v.W + px;
    if (kBlockMlp) {
        march_blocks_blend<DT>(a, v, recs, o, d, inv_d, omax, row);
        return;
    }
    RayState s = {{0.f, 0.f, 0.f}, {0.f, 0.f, 0.f, 0.f}, 1.f, 0, false};
    const int n_blk = v.ids_count;
    for (int k = 0; k < n_blk && !s.done; k++) march_block<DT>(recs[k], o, d, inv_d, omax, a.ert_eps, s, a.err);
    write_outputs(a, row, s, d, s_mlp);
}

// Thread schedule, block records in shared memory.
template <int DT, bool kBlockMlp>
__global__ void __launch_bounds__(kThreads, kMinBlocks) k_march_views(MarchArgs a) {
    __shared__ float s_mlp[kMlpParams + 1];
    extern __shared__ __align__(16) unsigned char s_dyn[];  // a.smem_recs block records
    BlockRec *s_rec = reinterpret_cast<BlockRec *>(s_dyn);
    __shared__ alignas(8) uint64_t s_bar;
    const int tile = blockIdx.x;
    const ViewRec &v = a.views[view_of_tile(a, tile)];
    const int n_blk = v.ids_count;
    const bool staged = n_blk > 0 && n_blk <= a.smem_recs;
    if (threadIdx.x == 0 && staged) mbar_init(&s_bar, 1);
    if (!kBlockMlp) load_mlp(a.mlp, s_mlp, (a.flags & 1u) != 0);
    __syncthreads();
    // the view's block records (near to far) go to shared memory by one TMA
    // bulk copy.  A wait that runs out records kErrTimeout and waits once more
    // (bounded) for the copy; if that also runs out the CTA leaves without
    // touching the records (the copy would then still be writing this CTA's
    // shared memory: two waits of 2^24 polls each, seconds, never seen short
    // of a stalled copy engine).
    if (staged) {
        const unsigned polls = a.wait_polls ? a.wait_polls : kWaitPolls;
        if (threadIdx.x == 0 && !(a.test_flags & kTestSkipRecordCopy))
            bulk_copy_g2s(s_rec, a.recs + v.ids_begin, (unsigned)(n_blk * sizeof(BlockRec)), &s_bar);
        if (!mbar_wait(&s_bar, 0, polls)) {
            atomicOr(a.err, kErrTimeout);
            if (!mbar_wait(&s_bar, 0, polls)) return;  // copy still in flight: leave without touching it
        }
    }
    march_tile_rays<DT, kBlockMlp>(a, v, staged ? s_rec : a.recs + v.ids_begin, tile, s_mlp);
}

// Thread schedule, block records in the launch's parameter buffer: the
// record fields the sample loop re-reads then come through the constant
// cache instead of taking shared-memory wavefronts from the L1 data pipe
// that the feature gathers are bound by.
template <int DT, bool kBlockMlp>
__global__ void __launch_bounds__(kThreads, kMinBlocks)
    k_march_views_c(const __grid_constant__ MarchArgs a, const __grid_constant__ ParamRecs pr) {
    __shared__ float s_mlp[kMlpParams + 1];
    const int tile = blockIdx.x;
    const ViewRec &v = a.views[view_of_tile(a, tile)];
    if (!kBlockMlp) {
        load_mlp(a.mlp, s_mlp, (a.flags & 1u) != 0);
        __syncthreads();
    }
    march_tile_rays<DT, kBlockMlp>(a, v, pr.r + v.ids_begin, tile, s_mlp);
}

// ---------------------------------------------------------------------------
// Warp-per-ray schedule.  A warp marches one ray at a time; lane l takes the
// lattice sample base + l, so the 32 gathers of one instruction read
// neighbouring texels of the same ray instead of 32 rays' far-apart texels.
// The in-block weights of Eq. 1 become an exclusive prefix product of
// exp(-sigma delta) across the lanes; the transmittance carried across chunks
// and blocks is Eq. 12-13.  Each lane finally owns one of the warp's 32 rays
// for the deferred MLP and the output writes.

__device__ __forceinline__ float warp_exclusive_product(float x, int lane, float &total) {
    float incl = x;
#pragma unroll
    for (int off = 1; off < 32; off <<= 1) {
        const float y = __shfl_up_sync(0xffffffffu, incl, off);
        if (lane >= off) incl *= y;
    }
    total = __shfl_sync(0xffffffffu, incl, 31);
    const float ex = __shfl_up_sync(0xffffffffu, incl, 1);
    return lane == 0 ? 1.0f : ex;
}

__device__ __forceinline__ float warp_sum(float x) {
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) x += __shfl_xor_sync(0xffffffffu, x, off);
    return x;
}

template <int DT>
__device__ __forceinline__ void march_block_warp(const BlockRec &b, const float o[3], const float d[3],
                                                 const float inv_d[3], float omax, float ert_eps, int lane,
                                                 float &T, float pc[3], float pf[4], int &nsamp, bool &done,
                                                 unsigned *err) {
    int i0, i1;
    float tfar;
    if (!candidate_range(b, o, d, inv_d, i0, i1, tfar)) return;
    if (i1 - i0 > kMaxSpan) {
        if (lane == 0) atomicOr(err, kErrRange);
        i1 = i0 + kMaxSpan;
    }
    const float delta = b.delta, inv_delta = 1.0f / b.delta;
    const float m = 4e-6f * (omax + tfar + b.bmax);
    const int Nc = b.Nc, C = b.C, R = b.R;
    for (int base = i0; base <= i1;) {
        const int i = base + lane;
        bool inb = false, occ = false;
        float p[3], g[3];
        int cell[3] = {0, 0, 0};
        if (i <= i1) {
            lattice_point(o, d, delta, i, p);
            inb = inside_block(b, p);
            if (inb) {
#pragma unroll
                for (int a = 0; a < 3; a++) {
                    g[a] = axis_coord(p[a], b.lo[a], b.kg[a]);
                    const int v = min(max(__float2int_rd(g[a]), 0), R - 2);
                    cell[a] = C == 1 ? v : (int)__umulhi((unsigned)v, b.cdiv);
                }
                const int ci = (cell[2] * Nc + cell[1]) * Nc + cell[0];
                occ = (__ldg(b.occ + (ci >> 5)) >> (ci & 31)) & 1u;
            }
        }
        float e = 1.f, c[7];
        if (occ) {
            float2 f2[4];
            BrickCache bc;  // one lattice sample of this lane: the brick is stored
            accumulate_sample<DT>(b, p, g, f2, &bc);
            const float f[8] = {f2[0].x, f2[0].y, f2[1].x, f2[1].y, f2[2].x, f2[2].y, f2[3].x, f2[3].y};
            e = __expf(-__expf(f[0]) * delta);
#pragma unroll
            for (int k = 0; k < 7; k++) c[k] = sigmoidf_fast(f[1 + k]);
        }
        float chunk;
        const float ex = warp_exclusive_product(e, lane, chunk);
        if (occ) {
            const float w = (T * ex) * (1.f - e);
#pragma unroll
            for (int k = 0; k < 3; k++) pc[k] = fmaf(w, c[k], pc[k]);
#pragma unroll
            for (int k = 0; k < 4; k++) pf[k] = fmaf(w, c[3 + k], pf[k]);
        }
        T *= chunk;
        nsamp += __popc(__ballot_sync(0xffffffffu, occ));
        // next chunk: past lane 31's empty cell when it sits in one (exact, as in the thread schedule)
        int j = -1;
        if (lane == 31 && inb && !occ) {
            float tx = 3.0e38f;
#pragma unroll
            for (int a = 0; a < 3; a++) {
                if (d[a] > 0.f) {
                    const float chi =
                        cell[a] == Nc - 1 ? b.hi[a] : fmaf((float)((cell[a] + 1) * C), b.vox[a], b.lo[a]);
                    tx = fminf(tx, (chi - m - o[a]) * inv_d[a]);
                } else if (d[a] < 0.f) {
                    const float clo = fmaf((float)(cell[a] * C), b.vox[a], b.lo[a]);
                    tx = fminf(tx, (clo + m - o[a]) * inv_d[a]);
                }
            }
            j = __float2int_rd(tx * inv_delta - 0.5f) - 1;
        }
        j = __shfl_sync(0xffffffffu, j, 31);
        base = max(base + 32, j + 1);
        if (T < ert_eps) {
            done = true;
            return;
        }
    }
}

template <int DT>
__global__ void __launch_bounds__(kThreads, kMinBlocksW) k_march_views_w(MarchArgs a) {
    __shared__ float s_mlp[kMlpParams + 1];
    __shared__ alignas(16) BlockRec s_rec[kMaxSmemRecs];
    __shared__ alignas(8) uint64_t s_bar;
    const int tile = blockIdx.x;
    const ViewRec &v = a.views[view_of_tile(a, tile)];
    const int n_blk = v.ids_count;
    const bool staged = n_blk > 0 && n_blk <= kMaxSmemRecs;
    if (threadIdx.x == 0 && staged) mbar_init(&s_bar, 1);
    load_mlp(a.mlp, s_mlp, (a.flags & 1u) != 0);
    __syncthreads();
    if (staged) {  // as in k_march_views
        const unsigned polls = a.wait_polls ? a.wait_polls : kWaitPolls;
        if (threadIdx.x == 0 && !(a.test_flags & kTestSkipRecordCopy))
            bulk_copy_g2s(s_rec, a.recs + v.ids_begin, (unsigned)(n_blk * sizeof(BlockRec)), &s_bar);
        if (!mbar_wait(&s_bar, 0, polls)) {
            atomicOr(a.err, kErrTimeout);
            if (!mbar_wait(&s_bar, 0, polls)) return;
        }
    }
    const BlockRec *recs = staged ? s_rec : a.recs + v.ids_begin;
    const int t = tile - v.tile_begin;
    int tx, ty;
    tile_xy(v, t, kTileH, tx, ty);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int px0 = tx * kTileW + (warp & 1) * 8, py0 = ty * kTileH + (warp >> 1) * 4;
    // this lane's own ray (it writes its outputs at the end)
    const int px = px0 + (lane & 7), py = py0 + (lane >> 3);
    const bool mine_valid = px < v.W && py < v.H;
    float mo[3], md[3];
    pixel_ray(v, min(px, v.W - 1), min(py, v.H - 1), mo, md);
    float my_acc[8] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 1.f};
    int my_n = 0;
    for (int q = 0; q < 32; q++) {
        const int qx = px0 + (q & 7), qy = py0 + (q >> 3);
        if (qx >= v.W || qy >= v.H) continue;  // uniform across the warp
        float o[3], d[3], inv_d[3], omax;
#pragma unroll
        for (int k = 0; k < 3; k++) {
            o[k] = __shfl_sync(0xffffffffu, mo[k], q);
            d[k] = __shfl_sync(0xffffffffu, md[k], q);
        }
        ray_setup(d, o, inv_d, omax);
        float T = 1.f, pc[3] = {0.f, 0.f, 0.f}, pf[4] = {0.f, 0.f, 0.f, 0.f};
        int nsamp = 0;
        bool done = false;
        for (int k = 0; k < n_blk && !done; k++)
            march_block_warp<DT>(recs[k], o, d, inv_d, omax, a.ert_eps, lane, T, pc, pf, nsamp, done, a.err);
        float tot[7];
#pragma unroll
        for (int k = 0; k < 3; k++) tot[k] = warp_sum(pc[k]);
#pragma unroll
        for (int k = 0; k < 4; k++) tot[3 + k] = warp_sum(pf[k]);
        if (lane == q) {
#pragma unroll
            for (int k = 0; k < 7; k++) my_acc[k] = tot[k];
            my_acc[7] = T;
            my_n = nsamp;
        }
    }
    if (!mine_valid) return;
    RayState s = {{my_acc[0], my_acc[1], my_acc[2]}, {my_acc[3], my_acc[4], my_acc[5], my_acc[6]}, my_acc[7], my_n,
                  false};
    write_outputs(a, v.pix_offset + (int64_t)py * v.W + px, s, md, s_mlp);
}

template <int DT, bool kBlockMlp>
__global__ void __launch_bounds__(kThreads, COW_RAYS_MIN_BLOCKS) k_march_rays(MarchArgs a,
                                                                          const __grid_constant__ RayRecs rr) {
    __shared__ float s_mlp[kMlpParams + 1];
    if (!kBlockMlp) {
        load_mlp(a.mlp, s_mlp, (a.flags & 1u) != 0);
        __syncthreads();
    }
    const int64_t t = (int64_t)blockIdx.x * kThreads + threadIdx.x;
    if (t >= a.n_rays) return;
    const int64_t r = a.ray_perm ? (int64_t)__ldg(a.ray_perm + t) : t;
    float o[3], d[3];
#pragma unroll
    for (int c = 0; c < 3; c++) {
        o[c] = __ldg(a.ray_o + 3 * r + c);
        d[c] = __ldg(a.ray_d + 3 * r + c);
    }
    // per-ray depth order: xy distance of block centres to this origin (App. D)
    int order[kMaxRayIds];
    const int n = sort_blocks_for_ray(rr, o, order);
    float inv_d[3], omax;
    ray_setup(d, o, inv_d, omax);
    if (kBlockMlp) {  // Eq. 5 with block id's own MLP at block_mlp_base + id * block_mlp_stride
        blend_blocks<DT>(
            a, n, [&](int k) -> const BlockRec & { return rr.r[order[k]]; },
            [&](int k) { return a.block_mlp_base + (int64_t)rr.id[order[k]] * a.block_mlp_stride; },
            [&](int k) -> float * {
                return a.out_block_state ? a.out_block_state + 8 * (r * rr.n + order[k]) : nullptr;
            },
            o, d, inv_d, omax, r);
        return;
    }
    RayState s = {{0.f, 0.f, 0.f}, {0.f, 0.f, 0.f, 0.f}, 1.f, 0, false};
    if (a.out_block_T) {
        // also every block's own transmittance, at its position in ids; -1
        // for a block without occupied samples (the call has no early
        // termination, so every block is marched)
        float *bt = a.out_block_T + r * n;
        for (int k = 0; k < n; k++) {
            float tb = 1.f;
            const int n0 = s.nsamp;
            march_block<DT>(rr.r[order[k]], o, d, inv_d, omax, a.ert_eps, s, a.err, &tb);
            bt[order[k]] = s.nsamp > n0 ? tb : -1.f;
        }
    } else {
        for (int k = 0; k < n && !s.done; k++)
            march_block<DT>(rr.r[order[k]], o, d, inv_d, omax, a.ert_eps, s, a.err);
    }
    write_outputs(a, r, s, d, s_mlp);
}

// Block-parallel form, first half: every block of the call marched on its
// own from an in-block transmittance of 1 (Eq. 11: C_d^k, F^k and T^k =
// 1 - alpha^k of block k alone), written as 8 floats per (ray, block) in
// the order of the call's ids.  No early termination (a partial must not
// depend on the blocks in front of it).
template <int DT>
__global__ void __launch_bounds__(kThreads, COW_RAYS_MIN_BLOCKS) k_march_partials(MarchArgs a,
                                                                              const __grid_constant__ RayRecs rr) {
    const int64_t t = (int64_t)blockIdx.x * kThreads + threadIdx.x;
    if (t >= a.n_rays) return;
    const int64_t r = a.ray_perm ? (int64_t)__ldg(a.ray_perm + t) : t;
    float o[3], d[3];
#pragma unroll
    for (int c = 0; c < 3; c++) {
        o[c] = __ldg(a.ray_o + 3 * r + c);
        d[c] = __ldg(a.ray_d + 3 * r + c);
    }
    float inv_d[3], omax;
    ray_setup(d, o, inv_d, omax);
    for (int k = 0; k < rr.n; k++) {
        RayState s = {{0.f, 0.f, 0.f}, {0.f, 0.f, 0.f, 0.f}, 1.f, 0, false};
        march_block<DT>(rr.r[k], o, d, inv_d, omax, 0.f, s, a.err);
        float4 *pp = reinterpret_cast<float4 *>(a.out_partials + 8 * (r * rr.n + k));
        pp[0] = make_float4(s.Cd[0], s.Cd[1], s.Cd[2], s.F[0]);
        pp[1] = make_float4(s.F[1], s.F[2], s.F[3], s.T);
    }
}

template <int DT, bool kBlockMlp>
cudaError_t launch_thread(const MarchArgs &a, int n_tiles, bool in_params, cudaStream_t st, const ParamRecs *pr) {
    if (in_params) {
        k_march_views_c<DT, kBlockMlp><<<n_tiles, kThreads, 0, st>>>(a, *pr);
    } else {
        // records staged in dynamic shared memory sized to the largest view's
        // list (the driver then sizes the shared-memory carveout for full
        // occupancy and leaves the rest of the SM's 256 KB to L1)
        const size_t smem = (size_t)a.smem_recs * sizeof(BlockRec);
        k_march_views<DT, kBlockMlp><<<n_tiles, kThreads, smem, st>>>(a);
    }
    return cudaGetLastError();
}

}  // namespace

// Per-dtype launchers (explicitly instantiated by march.cu for the dense
// grids and by march_bricks.cu for the brick-sparse ones).
template <int DT>
cudaError_t launch_views_dt(const MarchArgs &a, int n_tiles, int schedule, cudaStream_t st, const ParamRecs *pr) {
    const bool block_mlp = a.block_mlps != nullptr;
    if (schedule == kSchedWarp && !block_mlp) {
        k_march_views_w<DT><<<n_tiles, kThreads, 0, st>>>(a);
        return cudaGetLastError();
    }
    const bool in_params = schedule == kSchedThreadConst;
    if (in_params && !pr) return cudaErrorInvalidValue;
    return block_mlp ? launch_thread<DT, true>(a, n_tiles, in_params, st, pr)
                     : launch_thread<DT, false>(a, n_tiles, in_params, st, pr);
}

template <int DT>
cudaError_t launch_rays_dt(const MarchArgs &a, const RayRecs &rr, cudaStream_t st) {
    const int64_t nb = (a.n_rays + kThreads - 1) / kThreads;
    if (a.block_mlp_base) k_march_rays<DT, true><<<(unsigned)nb, kThreads, 0, st>>>(a, rr);
    else k_march_rays<DT, false><<<(unsigned)nb, kThreads, 0, st>>>(a, rr);
    return cudaGetLastError();
}

template <int DT>
cudaError_t launch_partials_dt(const MarchArgs &a, const RayRecs &rr, cudaStream_t st) {
    const int64_t nb = (a.n_rays + kThreads - 1) / kThreads;
    k_march_partials<DT><<<(unsigned)nb, kThreads, 0, st>>>(a, rr);
    return cudaGetLastError();
}

#define COW_INST_MARCH(D)                                                                                           \
    template cudaError_t launch_views_dt<(D)>(const MarchArgs &, int, int, cudaStream_t, const ParamRecs *);       \
    template cudaError_t launch_rays_dt<(D)>(const MarchArgs &, const RayRecs &, cudaStream_t);                    \
    template cudaError_t launch_partials_dt<(D)>(const MarchArgs &, const RayRecs &, cudaStream_t);

}  // namespace cow
