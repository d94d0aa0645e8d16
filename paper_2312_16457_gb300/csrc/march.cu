// march.cu -- the dense-grid variants of the view and ray marchers
// (march_kernels.cuh) and their dispatch by kernel dtype; march_bricks.cu
// holds the brick-sparse variants (separate translation units compile in
// parallel).
#include "march_kernels.cuh"

namespace cow {

COW_FOR_STORAGE(COW_INST_MARCH, 0)

#define COW_EXTERN_MARCH(D)                                                                                         \
    extern template cudaError_t launch_views_dt<(D)>(const MarchArgs &, int, int, cudaStream_t, const ParamRecs *); \
    extern template cudaError_t launch_rays_dt<(D)>(const MarchArgs &, const RayRecs &, cudaStream_t);
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

int march_tile_w() { return kTileW; }
int march_tile_h() { return kTileH; }

}  // namespace cow
