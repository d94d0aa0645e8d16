// kernel_launch.h -- per-dtype kernel launchers (internal to the library).
// Each is explicitly instantiated, for the dense or the brick-sparse DT
// values, in its own translation unit; the dispatchers pick one by the
// kernel dtype (storage | kBrickBit).
#pragma once

#include "cow_kernels.h"

namespace cow {

template <int DT>
cudaError_t launch_views_dt(const MarchArgs &a, int n_tiles, int schedule, cudaStream_t st, const ParamRecs *pr);
template <int DT>
cudaError_t launch_rays_dt(const MarchArgs &a, const RayRecs &rr, cudaStream_t st);
template <int DT>
cudaError_t launch_partials_dt(const MarchArgs &a, const RayRecs &rr, cudaStream_t st);
template <int DT>
cudaError_t launch_batch_smem_dt(const BatchArgs &a, int tile_cfg, int grid, cudaStream_t st);
template <int DT>
cudaError_t launch_batch_param_dt(const BatchArgs &a, int tile_cfg, int grid, cudaStream_t st, const ParamRecs *pr);

// F(storage | B) for every storage dtype
#define COW_FOR_STORAGE(F, B) F(kF32 | (B)) F(kF16 | (B)) F(kBF16 | (B)) F(kFP8 | (B)) F(kMixed | (B)) F(kFP8D | (B))

}  // namespace cow
