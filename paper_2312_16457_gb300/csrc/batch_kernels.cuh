// batch_kernels.cuh -- K8: persistent batched renderer over a (view, tile, block) work queue.
//
// Many cameras of uneven size and LOD set render in one launch: each CTA
// takes the next (view, tile) item from a device counter until the queue is
// empty.  A CTA loads the deferred MLP once, stages a view's block records
// into shared memory with a TMA bulk copy only when its item changes view,
// and culls that view's near-to-far block list against the tile's pyramid
// (the blocks whose grown box lies outside a plane through the camera and two
// neighbouring corner rays of the tile cannot contribute a sample to any of
// its rays) -- the tile x block decomposition.  The rays of the tile then
// march the culled list with the same per-ray code as the per-view kernel,
// so every pixel equals the per-view render bit for bit.
#pragma once

#include "cow_common.cuh"
#include "cow_kernels.h"
#include "kernel_launch.h"
#include "march_core.cuh"

namespace cow {

namespace {

#ifndef COW_BATCH_THREADS_PER_SM
#define COW_BATCH_THREADS_PER_SM 512
#endif

constexpr int kMaxBatchRecs = 96;             // block records a CTA stages
// resident threads per SM the register budget is sized for (128 registers a
// thread; measured faster than the compiler's own ~96-register choice)
constexpr int kBatchThreadsPerSm = COW_BATCH_THREADS_PER_SM;
constexpr unsigned kBatchWaitPolls = 1u << 24;  // bound on mbarrier polls

__device__ __forceinline__ void fence_proxy_async() {
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

// Unnormalised world direction through the centre of pixel (px, py).
__device__ __forceinline__ void corner_dir(const ViewRec &v, int px, int py, float w[3]) {
    const float xc = ((float)px + 0.5f - 0.5f * (float)v.W) / v.f;
    const float yc = -(((float)py + 0.5f - 0.5f * (float)v.H) / v.f);
#pragma unroll
    for (int r = 0; r < 3; r++) w[r] = v.Rm[3 * r] * xc + v.Rm[3 * r + 1] * yc - v.Rm[3 * r + 2];
}

// Cross product without fused multiply-adds: parallel inputs give exactly 0.
__device__ __forceinline__ void cross3(const float a[3], const float b[3], float c[3]) {
    c[0] = __fsub_rn(__fmul_rn(a[1], b[2]), __fmul_rn(a[2], b[1]));
    c[1] = __fsub_rn(__fmul_rn(a[2], b[0]), __fmul_rn(a[0], b[2]));
    c[2] = __fsub_rn(__fmul_rn(a[0], b[1]), __fmul_rn(a[1], b[0]));
}

__device__ __forceinline__ float norm1(const float a[3]) { return fabsf(a[0]) + fabsf(a[1]) + fabsf(a[2]); }

// True when the grown box of b is entirely on the outer side of one side
// plane of the tile pyramid (or behind the camera), by a margin above FP32
// error; such a block yields no lattice sample for any ray of the tile.
// Planes with use[k] == false (degenerate tiles: one pixel row or column)
// constrain nothing.
__device__ __forceinline__ bool culled(const BlockRec &b, const float o[3], const float n[4][3], const bool use[4],
                                       const float fwd[3]) {
    if (b.unb) return false;  // an unbounded block has no box to cull
    for (int k = 0; k < 5; k++) {
        if (k < 4 && !use[k]) continue;
        const float *nk = k < 4 ? n[k] : fwd;
        float pv[3];
#pragma unroll
        for (int a = 0; a < 3; a++) pv[a] = (nk[a] > 0.f ? b.hi_e[a] : b.lo_e[a]) - o[a];
        const float s = nk[0] * pv[0] + nk[1] * pv[1] + nk[2] * pv[2];
        const float mag = (fabsf(nk[0]) + fabsf(nk[1]) + fabsf(nk[2])) *
                          (fabsf(pv[0]) + fabsf(pv[1]) + fabsf(pv[2]));
        if (s < -1e-5f * mag) return true;
    }
    return false;
}

// Cull the view's n_blk records (near to far; rec_at(j) the j-th) against
// the pyramid of tile (tx, ty): s_list[0 .. *s_n) receives key(j) of the kept
// ones, in order.  Ends with a barrier.
// The side planes of the pyramid of tile (tx, ty) of TW x TH pixels (inward
// normals n, use[k] false for a degenerate side) and the view direction.
template <int TW, int TH>
__device__ __forceinline__ void tile_pyramid(const ViewRec &v, int tx, int ty, float n[4][3], bool use[4],
                                             float fwd[3]) {
    const int x0 = tx * TW, y0 = ty * TH;
    const int x1 = min(x0 + TW, v.W) - 1, y1 = min(y0 + TH, v.H) - 1;
    float c[4][3], ctr[3];
    fwd[0] = -v.Rm[2];
    fwd[1] = -v.Rm[5];
    fwd[2] = -v.Rm[8];
    corner_dir(v, x0, y0, c[0]);
    corner_dir(v, x1, y0, c[1]);
    corner_dir(v, x1, y1, c[2]);
    corner_dir(v, x0, y1, c[3]);
#pragma unroll
    for (int a3 = 0; a3 < 3; a3++) ctr[a3] = c[0][a3] + c[1][a3] + c[2][a3] + c[3][a3];
#pragma unroll
    for (int k = 0; k < 4; k++) {
        cross3(c[k], c[(k + 1) & 3], n[k]);
        // a plane is used only when its normal is well defined and the
        // tile's centre ray lies clearly on its inner side
        const float dn = n[k][0] * ctr[0] + n[k][1] * ctr[1] + n[k][2] * ctr[2];
        use[k] = norm1(n[k]) > 1e-5f * norm1(c[k]) * norm1(c[(k + 1) & 3]) &&
                 fabsf(dn) > 1e-4f * norm1(n[k]) * norm1(ctr);
        if (dn < 0.f) {
#pragma unroll
            for (int a3 = 0; a3 < 3; a3++) n[k][a3] = -n[k][a3];
        }
    }
}

template <int TW, int TH, class RecAt, class Key>
__device__ __forceinline__ void cull_tile(const ViewRec &v, int tx, int ty, int n_blk, RecAt rec_at, Key key,
                                          unsigned char *s_keep, short *s_list, int *s_n) {
    constexpr int kNT = TW * TH;
    float n[4][3], fwd[3];
    bool use[4];
    tile_pyramid<TW, TH>(v, tx, ty, n, use, fwd);
    for (int j = threadIdx.x; j < n_blk; j += kNT) s_keep[j] = culled(rec_at(j), v.o, n, use, fwd) ? 0 : 1;
    __syncthreads();
    if (threadIdx.x == 0) {
        int m = 0;
        for (int j = 0; j < n_blk; j++)
            if (s_keep[j]) s_list[m++] = (short)key(j);
        *s_n = m;
    }
    __syncthreads();
}

// March the rays of tile (tx, ty) through the records rec_by_key(s_list[k]),
// k < m, composite them and run the deferred MLP.
template <int DT, int TW, int TH, class RecByKey>
__device__ __forceinline__ void march_tile(const BatchArgs &a, const ViewRec &v, int tx, int ty, int m,
                                           const short *s_list, RecByKey rec_by_key, const float *s_mlp) {
    constexpr int kWarpsX = TW / 8;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int px = tx * TW + (warp % kWarpsX) * 8 + (lane & 7);
    const int py = ty * TH + (warp / kWarpsX) * 4 + (lane >> 3);
    if (px >= v.W || py >= v.H) return;
    float o[3], d[3], inv_d[3], omax;
    pixel_ray(v, px, py, o, d);
    ray_setup(d, o, inv_d, omax);
    RayState s = {{0.f, 0.f, 0.f}, {0.f, 0.f, 0.f, 0.f}, 1.f, 0, false};
    for (int k = 0; k < m && !s.done; k++) march_block<DT>(rec_by_key(s_list[k]), o, d, inv_d, omax, a.ert_eps, s, a.err);
    float x[10] = {s.Cd[0], s.Cd[1], s.Cd[2], s.F[0], s.F[1], s.F[2], s.F[3], d[0], d[1], d[2]};
    float out[3];
    deferred_mlp(s_mlp, x, (a.flags & 1u) != 0, out);
    const int64_t row = v.pix_offset + (int64_t)py * v.W + px;
    float *rgb = a.out_rgb + 3 * row;
    rgb[0] = s.Cd[0] + out[0];
    rgb[1] = s.Cd[1] + out[1];
    rgb[2] = s.Cd[2] + out[2];
    if (a.out_aux) {
        float4 *ap = reinterpret_cast<float4 *>(a.out_aux + 8 * row);
        ap[0] = make_float4(s.Cd[0], s.Cd[1], s.Cd[2], s.F[0]);
        ap[1] = make_float4(s.F[1], s.F[2], s.F[3], s.T);
    }
    if (a.out_nsamp) a.out_nsamp[row] = s.nsamp;
}

// The queue's bounds (hdr[0] views, hdr[1] items), read again for every item
// instead of held in registers across the march: the sample loop then keeps
// two more registers (at 16x8 tiles 73.8 -> 76.2 frames/s on one 1080p view).
__device__ __forceinline__ int queue_hdr(const BatchArgs &a, int k) { return *(volatile const int32_t *)(a.hdr + k); }

// View of an item: views are ordered by tile_begin.
__device__ __forceinline__ int view_of_item(const BatchArgs &a, int n_views, int item) {
    int lo = 0, hi = n_views - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (a.views[mid].tile_begin <= item) lo = mid;
        else hi = mid - 1;
    }
    return lo;
}

// Records staged in shared memory (or read from global memory for lists
// longer than kMaxBatchRecs).
template <int DT, int TW, int TH>
__global__ void __launch_bounds__(TW * TH, kBatchThreadsPerSm / (TW * TH)) k_march_batch(BatchArgs a) {
    __shared__ float s_mlp[kMlpParams + 1];
    extern __shared__ __align__(16) unsigned char s_dyn[];  // a.smem_recs block records
    BlockRec *s_rec = reinterpret_cast<BlockRec *>(s_dyn);
    __shared__ alignas(8) uint64_t s_bar;
    __shared__ int s_item, s_n;
    __shared__ unsigned char s_keep[kMaxBatchRecs];
    __shared__ short s_list[kMaxBatchRecs];
    if (threadIdx.x == 0) mbar_init(&s_bar, 1);
    load_mlp(a.mlp, s_mlp, (a.flags & 1u) != 0);
    __syncthreads();
    int cur_view = -1;
    unsigned phase = 0;
    bool staged = false;
    for (;;) {
        if (threadIdx.x == 0) s_item = (int)atomicAdd(a.counter, 1u);
        __syncthreads();
        const int item = s_item;
        if (item >= queue_hdr(a, 1)) break;
        const int vi = view_of_item(a, queue_hdr(a, 0), item);
        const ViewRec &v = a.views[vi];
        const int n_blk = v.ids_count;
        if (vi != cur_view) {
            cur_view = vi;
            staged = n_blk > 0 && n_blk <= a.smem_recs;
            if (staged) {
                // thread 0 copies and waits (bounded); the CTA then proceeds or
                // leaves as one, so no thread is left at a later barrier
                // (a second wait that also runs out leaves the copy possibly
                // still writing this CTA's shared memory: two waits of 2^24
                // polls, never seen short of a stalled copy engine)
                const unsigned polls = a.wait_polls ? a.wait_polls : kBatchWaitPolls;
                if (threadIdx.x == 0) {
                    fence_proxy_async();
                    if (!(a.test_flags & kTestSkipRecordCopy))
                        bulk_copy_g2s(s_rec, a.recs + v.ids_begin, (unsigned)(n_blk * sizeof(BlockRec)), &s_bar);
                    int ok = 1;
                    if (!mbar_wait(&s_bar, phase, polls)) {
                        atomicOr(a.err, kErrTimeout);
                        ok = mbar_wait(&s_bar, phase, polls) ? 1 : 0;
                    }
                    s_n = ok;
                }
                __syncthreads();
                if (!s_n) return;  // the copy never completed: every thread leaves
                mbar_wait(&s_bar, phase, polls);  // completed phase: returns at once, orders the reads
                phase ^= 1u;
            }
        }
        const BlockRec *recs = staged ? s_rec : a.recs + v.ids_begin;
        const int t = item - v.tile_begin;
        const int tx = t % v.tiles_x, ty = t / v.tiles_x;
        auto rec = [&](int j) -> const BlockRec & { return recs[j]; };
        if (n_blk <= kMaxBatchRecs) {
            // cull the view's blocks against the tile pyramid (order kept)
            cull_tile<TW, TH>(v, tx, ty, n_blk, rec, [](int j) { return j; }, s_keep, s_list, &s_n);
            march_tile<DT, TW, TH>(a, v, tx, ty, s_n, s_list, rec, s_mlp);
        } else {
            // too long to cull into shared memory: march the whole list
            if (threadIdx.x == 0) s_n = n_blk;
            for (int j = threadIdx.x; j < kMaxBatchRecs; j += TW * TH) s_list[j] = 0;
            __syncthreads();
            constexpr int kWarpsX = TW / 8;
            const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
            const int px = tx * TW + (warp % kWarpsX) * 8 + (lane & 7);
            const int py = ty * TH + (warp / kWarpsX) * 4 + (lane >> 3);
            if (px < v.W && py < v.H) {
                float o[3], d[3], inv_d[3], omax;
                pixel_ray(v, px, py, o, d);
                ray_setup(d, o, inv_d, omax);
                RayState s = {{0.f, 0.f, 0.f}, {0.f, 0.f, 0.f, 0.f}, 1.f, 0, false};
                for (int k = 0; k < n_blk && !s.done; k++)
                    march_block<DT>(recs[k], o, d, inv_d, omax, a.ert_eps, s, a.err);
                float x[10] = {s.Cd[0], s.Cd[1], s.Cd[2], s.F[0], s.F[1], s.F[2], s.F[3], d[0], d[1], d[2]};
                float out[3];
                deferred_mlp(s_mlp, x, (a.flags & 1u) != 0, out);
                const int64_t row = v.pix_offset + (int64_t)py * v.W + px;
                float *rgb = a.out_rgb + 3 * row;
                rgb[0] = s.Cd[0] + out[0];
                rgb[1] = s.Cd[1] + out[1];
                rgb[2] = s.Cd[2] + out[2];
                if (a.out_aux) {
                    float4 *ap = reinterpret_cast<float4 *>(a.out_aux + 8 * row);
                    ap[0] = make_float4(s.Cd[0], s.Cd[1], s.Cd[2], s.F[0]);
                    ap[1] = make_float4(s.F[1], s.F[2], s.F[3], s.T);
                }
                if (a.out_nsamp) a.out_nsamp[row] = s.nsamp;
            }
        }
        __syncthreads();  // s_item, s_list and s_rec are rewritten by the next item
    }
}

// A run of views whose distinct blocks fit the launch's parameter buffer:
// the records come by value (read through the constant cache, as in the
// per-view kernel, instead of taking shared-memory wavefronts from the L1
// data pipe the gathers are bound by); a view's near-to-far list is a list
// of indices into them (a.vidx + ids_begin).
template <int DT, int TW, int TH>
__global__ void __launch_bounds__(TW * TH, kBatchThreadsPerSm / (TW * TH))
    k_march_batch_c(const __grid_constant__ BatchArgs a, const __grid_constant__ ParamRecs pr) {
    __shared__ float s_mlp[kMlpParams + 1];
    __shared__ int s_item, s_n;
    __shared__ unsigned char s_keep[kParamRecs];
    __shared__ short s_list[kParamRecs];
    load_mlp(a.mlp, s_mlp, (a.flags & 1u) != 0);
    __syncthreads();
    for (;;) {
        if (threadIdx.x == 0) s_item = (int)atomicAdd(a.counter, 1u);
        __syncthreads();
        const int item = s_item;
        if (item >= queue_hdr(a, 1)) break;
        const ViewRec &v = a.views[view_of_item(a, queue_hdr(a, 0), item)];
        const int t = item - v.tile_begin;
        const int tx = t % v.tiles_x, ty = t / v.tiles_x;
        const unsigned char *idx = a.vidx + v.ids_begin;
        cull_tile<TW, TH>(
            v, tx, ty, v.ids_count, [&](int j) -> const BlockRec & { return pr.r[idx[j]]; },
            [&](int j) { return (int)idx[j]; }, s_keep, s_list, &s_n);
        march_tile<DT, TW, TH>(a, v, tx, ty, s_n, s_list, [&](int k) -> const BlockRec & { return pr.r[k]; }, s_mlp);
        __syncthreads();  // s_item and s_list are rewritten by the next item
    }
}

// Warp items: every warp takes its own 8x4-pixel item from the run's counter,
// culls the view's list against the item's pyramid with a ballot (the kept
// blocks as three 32-bit masks, near to far), and marches its 32 rays.  The
// loop has no CTA barrier, so a warp that finishes its item never waits for
// another warp of its CTA.  Records by value as k_march_batch_c.
constexpr int kWarpItemThreads = 128;

template <int DT>
__global__ void __launch_bounds__(kWarpItemThreads, kBatchThreadsPerSm / kWarpItemThreads)
    k_march_batch_w(const __grid_constant__ BatchArgs a, const __grid_constant__ ParamRecs pr) {
    static_assert(kParamRecs <= 96, "three 32-bit masks hold a run's lists");
    __shared__ float s_mlp[kMlpParams + 1];
    load_mlp(a.mlp, s_mlp, (a.flags & 1u) != 0);
    __syncthreads();
    const int lane = threadIdx.x & 31;
    for (;;) {
        int item = 0;
        if (lane == 0) item = (int)atomicAdd(a.counter, 1u);
        item = __shfl_sync(0xffffffffu, item, 0);
        if (item >= queue_hdr(a, 1)) break;
        const ViewRec &v = a.views[view_of_item(a, queue_hdr(a, 0), item)];
        const int t = item - v.tile_begin;
        const int tx = t % v.tiles_x, ty = t / v.tiles_x;
        const unsigned char *idx = a.vidx + v.ids_begin;
        const int n_blk = v.ids_count;
        unsigned keep[3];
        {
            float n[4][3], fwd[3];
            bool use[4];
            tile_pyramid<8, 4>(v, tx, ty, n, use, fwd);
#pragma unroll
            for (int w = 0; w < 3; w++) {
                const int j = 32 * w + lane;
                const bool k = j < n_blk && !culled(pr.r[__ldg(idx + j)], v.o, n, use, fwd);
                keep[w] = __ballot_sync(0xffffffffu, k);
            }
        }
        const int px = tx * 8 + (lane & 7), py = ty * 4 + (lane >> 3);
        if (px < v.W && py < v.H) {  // lanes off the image idle until the next item
            float o[3], d[3], inv_d[3], omax;
            pixel_ray(v, px, py, o, d);
            ray_setup(d, o, inv_d, omax);
            const int64_t row = v.pix_offset + (int64_t)py * v.W + px;
            RayState s = {{0.f, 0.f, 0.f}, {0.f, 0.f, 0.f, 0.f}, 1.f, 0, false};
            for (int w = 0; w < 3 && !s.done; w++) {
                unsigned m = keep[w];
                while (m && !s.done) {
                    const int j = 32 * w + __ffs(m) - 1;
                    m &= m - 1;
                    march_block<DT>(pr.r[__ldg(idx + j)], o, d, inv_d, omax, a.ert_eps, s, a.err);
                }
            }
            float x[10] = {s.Cd[0], s.Cd[1], s.Cd[2], s.F[0], s.F[1], s.F[2], s.F[3], d[0], d[1], d[2]};
            float out[3];
            deferred_mlp(s_mlp, x, (a.flags & 1u) != 0, out);
            float *rgb = a.out_rgb + 3 * row;
            rgb[0] = s.Cd[0] + out[0];
            rgb[1] = s.Cd[1] + out[1];
            rgb[2] = s.Cd[2] + out[2];
            if (a.out_aux) {
                float4 *ap = reinterpret_cast<float4 *>(a.out_aux + 8 * row);
                ap[0] = make_float4(s.Cd[0], s.Cd[1], s.Cd[2], s.F[0]);
                ap[1] = make_float4(s.F[1], s.F[2], s.F[3], s.T);
            }
            if (a.out_nsamp) a.out_nsamp[row] = s.nsamp;
        }
    }
}

}  // namespace

// Per-dtype launchers: records staged in shared memory (batch.cu, dense;
// batch_bricks.cu) or by value in the parameter buffer (batch_param.cu,
// batch_param_bricks.cu).
template <int DT>
cudaError_t launch_batch_smem_dt(const BatchArgs &a, int tile_cfg, int grid, cudaStream_t st) {
    const size_t smem = (size_t)a.smem_recs * sizeof(BlockRec);
    switch (tile_cfg) {
    case 0: k_march_batch<DT, 16, 8><<<grid, 128, smem, st>>>(a); break;
    case 1: k_march_batch<DT, 8, 8><<<grid, 64, smem, st>>>(a); break;
    case 2: k_march_batch<DT, 16, 16><<<grid, 256, smem, st>>>(a); break;
    case 3: k_march_batch<DT, 32, 8><<<grid, 256, smem, st>>>(a); break;
    default: return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
}

template <int DT>
cudaError_t launch_batch_param_dt(const BatchArgs &a, int tile_cfg, int grid, cudaStream_t st, const ParamRecs *pr) {
    switch (tile_cfg) {
    case 0: k_march_batch_c<DT, 16, 8><<<grid, 128, 0, st>>>(a, *pr); break;
    case 1: k_march_batch_c<DT, 8, 8><<<grid, 64, 0, st>>>(a, *pr); break;
    case 2: k_march_batch_c<DT, 16, 16><<<grid, 256, 0, st>>>(a, *pr); break;
    case 3: k_march_batch_c<DT, 32, 8><<<grid, 256, 0, st>>>(a, *pr); break;
    case 4: k_march_batch_w<DT><<<grid, kWarpItemThreads, 0, st>>>(a, *pr); break;
    default: return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
}

#define COW_INST_BATCH_SMEM(D) \
    template cudaError_t launch_batch_smem_dt<(D)>(const BatchArgs &, int, int, cudaStream_t);
#define COW_INST_BATCH_PARAM(D) \
    template cudaError_t launch_batch_param_dt<(D)>(const BatchArgs &, int, int, cudaStream_t, const ParamRecs *);

}  // namespace cow
