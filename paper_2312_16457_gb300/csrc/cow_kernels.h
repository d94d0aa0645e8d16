// cow_kernels.h -- launch interfaces of the libcow kernels (internal to the library).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace cow {

struct BlockRec;
struct ViewRec;

struct MarchArgs {
    const BlockRec *recs;  // view mode: the views' block records, near to far, by ViewRec::ids_begin;
                           // ray mode: every block of the context, indexed by ids
    const ViewRec *views;
    int32_t n_views;
    int32_t dtype;
    const int32_t *ids;    // ray mode: the blocks to composite
    const float *mlp;      // 499 FP32 (device)
    float ert_eps;
    uint32_t flags;
    float *out_rgb;
    float *out_aux;        // may be null
    int32_t *out_nsamp;    // may be null
    unsigned *err;
    const float *ray_o;    // ray mode
    const float *ray_d;
    int64_t n_rays;
    int32_t n_ray_ids;
};

// marching schedules of the view kernel
constexpr int kSchedWarp = 0;    // one ray per warp, lanes on consecutive lattice samples
constexpr int kSchedThread = 1;  // one ray per thread
cudaError_t launch_march_views(const MarchArgs &a, int n_tiles, int schedule, cudaStream_t st);
cudaError_t launch_march_rays(const MarchArgs &a, cudaStream_t st);
int march_tile_w();
int march_tile_h();

// K4 / K5: packing and occupancy (pack.cu)
cudaError_t launch_amax8(const float *x, int64_t n_vec, unsigned *amax_bits, cudaStream_t st);
// FP32 packs in the natural layout; FP16 / BF16 / FP8 in the pair layout
// (element i = vertex i and vertex i+1 of its row of `row` vertices).
cudaError_t launch_pack(const float *x, int64_t n_vec, int row, int dtype, const float *inv_scale8, void *out,
                        cudaStream_t st);
cudaError_t launch_occupancy(const float *grid, int R, int C, double log_thresh, uint32_t *bits, cudaStream_t st);

}  // namespace cow
