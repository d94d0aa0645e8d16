// batch.cu -- the batched form's dense-grid kernels with shared-memory
// records (batch_kernels.cuh) and the dispatch of every variant by kernel
// dtype and record placement; the other variants live in batch_bricks.cu,
// batch_param.cu and batch_param_bricks.cu (translation units that compile
// in parallel).
#include "batch_kernels.cuh"

namespace cow {

COW_FOR_STORAGE(COW_INST_BATCH_SMEM, 0)

#define COW_EXTERN_BATCH(D)                                                                                     \
    extern template cudaError_t launch_batch_smem_dt<(D)>(const BatchArgs &, int, int, cudaStream_t);          \
    extern template cudaError_t launch_batch_param_dt<(D)>(const BatchArgs &, int, int, cudaStream_t,          \
                                                           const ParamRecs *);
COW_FOR_STORAGE(COW_EXTERN_BATCH, kBrickBit)
#define COW_EXTERN_BATCH_PARAM(D) \
    extern template cudaError_t launch_batch_param_dt<(D)>(const BatchArgs &, int, int, cudaStream_t, const ParamRecs *);
COW_FOR_STORAGE(COW_EXTERN_BATCH_PARAM, 0)

// tile_cfg 4: 8x4 pixels per warp (warp items, records by value only).
void batch_tile_shape(int tile_cfg, int *tw, int *th) {
    static const int s[5][2] = {{16, 8}, {8, 8}, {16, 16}, {32, 8}, {8, 4}};
    const int k = tile_cfg < 0 || tile_cfg > 4 ? 0 : tile_cfg;
    *tw = s[k][0];
    *th = s[k][1];
}

cudaError_t launch_march_batch(const BatchArgs &a, int tile_cfg, int grid, cudaStream_t st, const ParamRecs *pr) {
    return dispatch_dt(a.dtype, [&](auto D) {
        return pr ? launch_batch_param_dt<decltype(D)::value>(a, tile_cfg, grid, st, pr)
                  : launch_batch_smem_dt<decltype(D)::value>(a, tile_cfg, grid, st);
    });
}

}  // namespace cow
