// ray_order.cu -- a coherent processing order for ray batches.
//
// The ray-batch form (training rays: origins and directions in any order)
// marches one ray per thread.  When neighbouring threads hold unrelated
// rays, every gather of a warp lands on a different texel line and the
// forward and backward re-march run several times slower than on a camera's
// coherent rays.  The order below groups rays that enter the call's blocks
// near one another, in a similar direction: key = Morton code of the entry
// point's cell on an 8 x 8 x 8 grid over the blocks' bounding box, then the
// direction's cell on an 8 x 8 x 8 grid over [-1, 1]^3, and a counting sort
// of the keys gives the permutation the ray kernels read (thread t marches
// ray perm[t]; every output stays at its ray's own index, so the results
// per ray do not depend on the order).
#include <algorithm>

#include "cow_common.cuh"
#include "cow_kernels.h"

namespace cow {

namespace {

constexpr int kCellBits = 3;   // 8 cells per axis of the entry point
constexpr int kDirBits = 3;    // 8 cells per direction component
static_assert(3 * kCellBits + 3 * kDirBits == kRayOrderKeyBits, "key width");

__device__ __forceinline__ uint32_t spread3(uint32_t v) {  // bit i -> bit 3 i (v < 2^kCellBits)
    uint32_t r = 0;
#pragma unroll
    for (int i = 0; i < kCellBits; i++) r |= ((v >> i) & 1u) << (3 * i);
    return r;
}

__device__ __forceinline__ uint32_t cell_of(float x, float lo, float inv_ext, int bits) {
    const float n = (float)(1 << bits);
    const float q = fminf(fmaxf((x - lo) * inv_ext * n, 0.f), n - 1.f);  // NaN -> 0
    return (uint32_t)q;
}

__global__ void k_ray_keys(const float *__restrict__ o, const float *__restrict__ d, int64_t n, float3 lo, float3 hi,
                           uint32_t *__restrict__ keys, uint32_t *__restrict__ hist) {
    const float3 inv = make_float3(1.f / fmaxf(hi.x - lo.x, 1e-30f), 1.f / fmaxf(hi.y - lo.y, 1e-30f),
                                   1.f / fmaxf(hi.z - lo.z, 1e-30f));
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const float oo[3] = {o[3 * i], o[3 * i + 1], o[3 * i + 2]};
        const float dd[3] = {d[3 * i], d[3 * i + 1], d[3 * i + 2]};
        const float l[3] = {lo.x, lo.y, lo.z}, h[3] = {hi.x, hi.y, hi.z};
        // entry point into the box (the origin itself when inside or behind)
        float tn = 0.f;
#pragma unroll
        for (int a = 0; a < 3; a++) {
            if (dd[a] == 0.f) continue;
            const float t1 = (l[a] - oo[a]) / dd[a], t2 = (h[a] - oo[a]) / dd[a];
            tn = fmaxf(tn, fminf(t1, t2));
        }
        const float p[3] = {oo[0] + tn * dd[0], oo[1] + tn * dd[1], oo[2] + tn * dd[2]};
        const float iv[3] = {inv.x, inv.y, inv.z};
        uint32_t m = 0, dc = 0;
#pragma unroll
        for (int a = 0; a < 3; a++) {
            m |= spread3(cell_of(p[a], l[a], iv[a], kCellBits)) << a;
            dc = (dc << kDirBits) | cell_of(dd[a], -1.f, 0.5f, kDirBits);
        }
        const uint32_t key = (m << (3 * kDirBits)) | dc;
        keys[i] = key;
        atomicAdd(hist + key, 1u);
    }
}

// Exclusive prefix sum of the kRayOrderBins counts in two levels: every CTA
// scans its kScanThreads bins in place and writes its total to sums[]; one
// CTA then scans the totals, which the scatter adds back.
constexpr int kScanThreads = 1024;
constexpr int kScanBlocks = kRayOrderBins / kScanThreads;

__device__ __forceinline__ uint32_t block_exclusive_scan(uint32_t v, uint32_t *s_warp, uint32_t *total) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    uint32_t x = v;
#pragma unroll
    for (int off = 1; off < 32; off <<= 1) {
        const uint32_t y = __shfl_up_sync(0xffffffffu, x, off);
        if (lane >= off) x += y;
    }
    if (lane == 31) s_warp[warp] = x;
    __syncthreads();
    if (warp == 0) {
        const int nw = blockDim.x >> 5;
        uint32_t w = lane < nw ? s_warp[lane] : 0u;
#pragma unroll
        for (int off = 1; off < 32; off <<= 1) {
            const uint32_t y = __shfl_up_sync(0xffffffffu, w, off);
            if (lane >= off) w += y;
        }
        if (lane < nw) s_warp[lane] = w;  // inclusive warp totals
    }
    __syncthreads();
    if (total) *total = s_warp[(blockDim.x >> 5) - 1];
    return x - v + (warp > 0 ? s_warp[warp - 1] : 0u);
}

__global__ void __launch_bounds__(kScanThreads) k_scan_local(uint32_t *hist, uint32_t *sums) {
    __shared__ uint32_t s_warp[32];
    const int64_t i = (int64_t)blockIdx.x * kScanThreads + threadIdx.x;
    uint32_t total;
    const uint32_t ex = block_exclusive_scan(hist[i], s_warp, &total);
    hist[i] = ex;
    if (threadIdx.x == 0) sums[blockIdx.x] = total;
}

__global__ void __launch_bounds__(kScanBlocks) k_scan_sums(uint32_t *sums) {
    __shared__ uint32_t s_warp[32];
    sums[threadIdx.x] = block_exclusive_scan(sums[threadIdx.x], s_warp, nullptr);
}

__global__ void k_ray_scatter(const uint32_t *__restrict__ keys, int64_t n, uint32_t *__restrict__ offs,
                              const uint32_t *__restrict__ sums, int32_t *__restrict__ perm) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const uint32_t k = keys[i];
        perm[sums[k / kScanThreads] + atomicAdd(offs + k, 1u)] = (int32_t)i;
    }
}

}  // namespace

cudaError_t launch_ray_order(const float *o, const float *d, int64_t n, const float lo[3], const float hi[3],
                             uint32_t *keys, uint32_t *hist, int32_t *perm, cudaStream_t st) {
    static_assert(kRayOrderBins == kScanBlocks * kScanThreads && kScanBlocks <= 1024 && kScanBlocks % 32 == 0,
                  "two-level scan shape");
    static_assert(kRayOrderHistWords == kRayOrderBins + kScanBlocks, "histogram scratch: bins, then block totals");
    if (n <= 0 || n > 0x7fffffff) return cudaErrorInvalidValue;
    cudaError_t e = cudaMemsetAsync(hist, 0, kRayOrderBins * sizeof(uint32_t), st);
    if (e != cudaSuccess) return e;
    uint32_t *sums = hist + kRayOrderBins;
    const int grid = (int)std::min<int64_t>((n + 255) / 256, 152 * 16);
    k_ray_keys<<<grid, 256, 0, st>>>(o, d, n, make_float3(lo[0], lo[1], lo[2]), make_float3(hi[0], hi[1], hi[2]), keys,
                                     hist);
    k_scan_local<<<kScanBlocks, kScanThreads, 0, st>>>(hist, sums);
    k_scan_sums<<<1, kScanBlocks, 0, st>>>(sums);
    k_ray_scatter<<<grid, 256, 0, st>>>(keys, n, hist, sums, perm);
    return cudaGetLastError();
}

}  // namespace cow
