// march.cu -- the dense-grid variants of the view and ray marchers
// (march_kernels.cuh) and their dispatch by kernel dtype; march_bricks.cu
// holds the brick-sparse variants (separate translation units compile in
// parallel).
#include "march_kernels.cuh"

namespace cow {

COW_FOR_STORAGE(COW_INST_MARCH, 0)

#define COW_EXTERN_MARCH(D)                                                                                         \
    extern template cudaError_t launch_views_dt<(D)>(const MarchArgs &, int, int, cudaStream_t, const ParamRecs *); \
    extern template cudaError_t launch_rays_dt<(D)>(const MarchArgs &, const RayRecs &, cudaStream_t);              \
    extern template cudaError_t launch_partials_dt<(D)>(const MarchArgs &, const RayRecs &, cudaStream_t);
COW_FOR_STORAGE(COW_EXTERN_MARCH, kBrickBit)

cudaError_t launch_march_views(const MarchArgs &a, int n_tiles, int schedule, cudaStream_t st,
                               const ParamRecs *pr) {
    if (n_tiles <= 0) return cudaSuccess;
    return dispatch_dt(a.dtype,
                       [&](auto D) { return launch_views_dt<decltype(D)::value>(a, n_tiles, schedule, st, pr); });
}

cudaError_t launch_march_rays(const MarchArgs &a, const RayRecs &rr, cudaStream_t st) {
    if (a.n_rays <= 0) return cudaSuccess;
    return dispatch_dt(a.dtype, [&](auto D) { return launch_rays_dt<decltype(D)::value>(a, rr, st); });
}

cudaError_t launch_march_partials(const MarchArgs &a, const RayRecs &rr, cudaStream_t st) {
    if (a.n_rays <= 0) return cudaSuccess;
    return dispatch_dt(a.dtype, [&](auto D) { return launch_partials_dt<decltype(D)::value>(a, rr, st); });
}

namespace {

// K2, the block-parallel form's second half: per ray, the partials of its
// blocks folded near to far with the "over" of Eq. 12-13,
//   (C, F, T) <- (C + T C^k, F + T F^k, T T^k),
// in the ray's own depth order (App. D key from its origin, as the ray
// form), then the deferred MLP (Eq. 3).
__global__ void __launch_bounds__(kThreads) k_composite_over(MarchArgs a, const __grid_constant__ RayRecs rr) {
    __shared__ float s_mlp[kMlpParams + 1];
    load_mlp(a.mlp, s_mlp, (a.flags & 1u) != 0);
    __syncthreads();
    const int64_t r = (int64_t)blockIdx.x * kThreads + threadIdx.x;
    if (r >= a.n_rays) return;
    float o[3], d[3];
#pragma unroll
    for (int c = 0; c < 3; c++) {
        o[c] = __ldg(a.ray_o + 3 * r + c);
        d[c] = __ldg(a.ray_d + 3 * r + c);
    }
    int order[kMaxRayIds];
    const int n = sort_blocks_for_ray(rr, o, order);
    RayState s = {{0.f, 0.f, 0.f}, {0.f, 0.f, 0.f, 0.f}, 1.f, 0, false};
    for (int k = 0; k < n; k++) {
        const float4 *pp = reinterpret_cast<const float4 *>(a.in_partials + 8 * (r * rr.n + order[k]));
        const float4 p0 = __ldg(pp), p1 = __ldg(pp + 1);
        s.Cd[0] = fmaf(s.T, p0.x, s.Cd[0]);
        s.Cd[1] = fmaf(s.T, p0.y, s.Cd[1]);
        s.Cd[2] = fmaf(s.T, p0.z, s.Cd[2]);
        s.F[0] = fmaf(s.T, p0.w, s.F[0]);
        s.F[1] = fmaf(s.T, p1.x, s.F[1]);
        s.F[2] = fmaf(s.T, p1.y, s.F[2]);
        s.F[3] = fmaf(s.T, p1.z, s.F[3]);
        s.T *= p1.w;
    }
    float x[10] = {s.Cd[0], s.Cd[1], s.Cd[2], s.F[0], s.F[1], s.F[2], s.F[3], d[0], d[1], d[2]};
    float out[3];
    deferred_mlp(s_mlp, x, (a.flags & 1u) != 0, out);
    float *rgb = a.out_rgb + 3 * r;
    rgb[0] = s.Cd[0] + out[0];
    rgb[1] = s.Cd[1] + out[1];
    rgb[2] = s.Cd[2] + out[2];
    if (a.out_aux) {
        float4 *ap = reinterpret_cast<float4 *>(a.out_aux + 8 * r);
        ap[0] = make_float4(s.Cd[0], s.Cd[1], s.Cd[2], s.F[0]);
        ap[1] = make_float4(s.F[1], s.F[2], s.F[3], s.T);
    }
}

}  // namespace

cudaError_t launch_composite_over(const MarchArgs &a, const RayRecs &rr, cudaStream_t st) {
    if (a.n_rays <= 0) return cudaSuccess;
    const int64_t nb = (a.n_rays + kThreads - 1) / kThreads;
    k_composite_over<<<(unsigned)nb, kThreads, 0, st>>>(a, rr);
    return cudaGetLastError();
}

int march_tile_w() { return kTileW; }
int march_tile_h() { return kTileH; }

}  // namespace cow
