// cow_kernels.h -- launch interfaces of the libcow kernels (internal to the library).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace cow {

struct BlockRec;
struct ViewRec;
struct RayRecs;

struct MarchArgs {
    const BlockRec *recs;  // view mode: the views' block records, near to far, by ViewRec::ids_begin
                           // (ray mode takes its records by value, RayRecs)
    const ViewRec *views;
    int32_t n_views;
    int32_t dtype;
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
    int32_t smem_recs;     // view mode, thread schedule: block records the launch's shared memory holds
    const float *const *block_mlps;  // view mode, per-block MLPs: weights of record k, parallel to recs
    int32_t n_freq;                  // PE frequencies of the per-block MLPs
    float *out_block_T;              // ray mode, may be null: n_rays x n_ray_ids in-block transmittances
    const float *block_mlp_base;     // ray mode, per-block MLPs: block id's weights at base + id * stride
    int64_t block_mlp_stride;        // floats (null base: the global MLP)
    uint32_t test_flags;             // kTestSkipRecordCopy (tests of the bounded waits); 0 in production
    uint32_t wait_polls;             // bound on each mbarrier wait (0: the kernel's default)
    float *out_partials;             // block-parallel form: n_rays x n_ids x 8 per-block partials (written)
    const float *in_partials;        // block-parallel form: the same, read by the compositor
    const int32_t *ray_perm;         // ray mode, may be null: thread t marches ray ray_perm[t] (outputs at the ray's index)
    float *out_block_state;          // ray mode, per-block MLPs, may be null: n_rays x n_ids x 8, per (ray, block
                                     // at its position in ids) C^k (3), F^k (4), the transmittance in front (-1: no sample)
};

// Test hook of the kernels that stage block records with a TMA bulk copy:
// the copy is not issued, so the barrier's phase never completes and the
// bounded wait runs out with nothing in flight.
constexpr uint32_t kTestSkipRecordCopy = 1u;

// marching schedules of the view kernel
constexpr int kSchedWarp = 0;         // one ray per warp, lanes on consecutive lattice samples
constexpr int kSchedThread = 1;       // one ray per thread, records in shared memory
constexpr int kSchedThreadConst = 2;  // one ray per thread, records in the parameter buffer
struct ParamRecs;
cudaError_t launch_march_views(const MarchArgs &a, int n_tiles, int schedule, cudaStream_t st,
                               const ParamRecs *pr = nullptr);
cudaError_t launch_march_rays(const MarchArgs &a, const RayRecs &rr, cudaStream_t st);
// A coherent order of a ray batch (ray_order.cu): perm[t] = the ray thread t
// marches, grouping rays by the cell of their entry into the box [lo, hi]
// and of their direction.  keys: n scratch words; hist: kRayOrderHistWords
// words (the bins, then the totals of the scan's blocks of 1024 bins).
constexpr int kRayOrderKeyBits = 18;
constexpr int kRayOrderBins = 1 << kRayOrderKeyBits;
constexpr int kRayOrderHistWords = kRayOrderBins + kRayOrderBins / 1024;
cudaError_t launch_ray_order(const float *o, const float *d, int64_t n, const float lo[3], const float hi[3],
                             uint32_t *keys, uint32_t *hist, int32_t *perm, cudaStream_t st);
// Block-parallel form: per-block partials of a ray batch (8 floats per ray
// and block, in the order of rr), and K2, their near-to-far "over" with the
// deferred MLP (Eq. 12-13, Eq. 3).
cudaError_t launch_march_partials(const MarchArgs &a, const RayRecs &rr, cudaStream_t st);
cudaError_t launch_composite_over(const MarchArgs &a, const RayRecs &rr, cudaStream_t st);
int march_tile_w();
int march_tile_h();

// K6 / K7: gradients of the ray-batch form (bwd.cu)
struct BwdArgs {                  // the call's block records come by value (RayRecs)
    int32_t dtype;
    const float *mlp;             // 499 FP32 (device)
    float ert_eps;
    const float *ray_o, *ray_d;   // n_rays x 3
    int64_t n_rays;
    const float *aux;             // forward aux, n_rays x 8
    const float *dL_drgb;         // n_rays x 3
    float *const *grad_grid;      // device array of per-block pointers (entries may be null)
    float *const *grad_planes;    // device array of 3 per-block pointers
    float *grad_mlp;              // 499, accumulated
    float *partials;              // scratch: backward_rows(n_rays) x 499
    float *gcf;                   // scratch: n_rays x 8 (dL/dC_d, dL/dF per ray)
    unsigned *err;
    const int32_t *ray_perm;      // may be null: the re-march's thread t takes ray ray_perm[t]
};

// Gradients of the ray-batch form with per-block MLPs (Eq. 5), bwd.cu
struct BmBwdArgs {                // the call's block records come by value (RayRecs)
    int32_t dtype;
    const float *ray_o, *ray_d;   // n_rays x 3
    int64_t n_rays;
    const float *dL_drgb;         // n_rays x 3
    float *const *grad_grid;      // device array of per-block pointers (entries may be null)
    float *const *grad_planes;    // device array of 3 per-block pointers
    const float *mlps;            // block i's weights at mlps + i * mlp_stride (the context's copy)
    int64_t mlp_stride;
    float *grad_mlps;             // block i's weight gradient at grad_mlps + i * grad_stride (accumulated)
    int64_t grad_stride;
    int32_t n_freq;
    int32_t n_ids;
    float *S;                     // scratch n_rays x n_ids x 8: C^k (3), F^k (4), B_k (-1: no sample)
    float *G;                     // scratch n_rays x n_ids x 8: dL/dC^k (3), dL/dF^k (4), dL/dC . X_k
    unsigned *err;
    const int32_t *ray_perm;      // may be null: the marching passes' thread t takes ray ray_perm[t]
    int32_t have_state;           // S already holds the forward's per-block state: skip the first pass
};
cudaError_t launch_backward_block_mlps(const BmBwdArgs &a, const RayRecs &rr, cudaStream_t st);

// Training-stage regularisers (bwd.cu): sparsity (Eq. 7) over points,
// block opacity (Eq. 8) over rays
struct RegArgs {                  // the blocks that take part come by value (RayRecs)
    int32_t dtype;
    const float *pts;             // sparsity: n x 3 points
    const float *ray_o, *ray_d;   // opacity: n x 3 rays
    int64_t n;
    float weight;                 // the loss and its gradient are scaled by weight / n
    const float *block_T;         // opacity: the forward's n x n_ids in-block transmittances (-1: no
                                  // sample), or null to march every block twice
    float *loss;                  // device float, accumulated (may be null)
    float *const *grad_grid;      // device pointer table as in BwdArgs (null: no gradient)
    float *const *grad_planes;
    unsigned *err;
    const int32_t *ray_perm;      // opacity, may be null: thread t takes ray ray_perm[t]
};
cudaError_t launch_sparsity(const RegArgs &a, const RayRecs &rr, cudaStream_t st);
cudaError_t launch_opacity(const RegArgs &a, const RayRecs &rr, cudaStream_t st);
// threads per CTA of the backward kernels: one MLP-gradient scratch row per
// CTA, backward_rows(n) = ceil(n / kBwdCtaThreads)
constexpr int kBwdCtaThreads = 128;
int backward_rows(int64_t n_rays);
cudaError_t launch_backward_rays(const BwdArgs &a, const RayRecs &rr, cudaStream_t st);
cudaError_t launch_adam(float *p, const float *g, float *m, float *v, int64_t n, float lr, float b1, float b2,
                        float eps, int step, cudaStream_t st);
cudaError_t launch_mse_grad(const float *rgb, const float *tgt, int64_t n, float *grad, float *loss, cudaStream_t st);

// FP64 render of ray batches for finite-difference checks (check_f64.cu):
// the FP32 marcher's samples, every value after them in FP64 from FP64
// copies of the features (device tables of per-block pointers by block id).
struct F64Args {
    const float *ray_o, *ray_d;   // n_rays x 3 (device)
    int64_t n_rays;
    const double *const *grids;   // [block id] -> R^3 x 8 FP64
    const double *const *planes;  // [3 id + k] -> P^2 x 8 FP64
    const double *mlp;            // 499 FP64
    double *out_rgb;              // n_rays x 3
    double *out_aux;              // n_rays x 8 (may be null): C_d, F, T
    unsigned *err;
};
cudaError_t launch_march_rays_f64(const F64Args &a, const RayRecs &rr, cudaStream_t st);

// K8: persistent batched renderer (batch.cu)
struct BatchArgs {
    const int32_t *hdr;      // device: n_views, n_items (tiles of all views)
    const ViewRec *views;    // tile_begin ascending
    const BlockRec *recs;    // the views' block records, near to far, by ViewRec::ids_begin
    const float *mlp;        // 499 FP32 (device)
    float ert_eps;
    uint32_t flags;
    int32_t dtype;
    int32_t smem_recs;       // block records the launch's dynamic shared memory holds (0: read from global)
    float *out_rgb;
    float *out_aux;          // may be null
    int32_t *out_nsamp;      // may be null
    unsigned *err;
    unsigned *counter;       // work-queue head, zero at launch
    uint32_t test_flags;     // kTestSkipRecordCopy (tests of the bounded waits); 0 in production
    uint32_t wait_polls;     // bound on each mbarrier wait (0: the kernel's default)
    const unsigned char *vidx;  // records by value (pr): each view's list as indices into them, by ids_begin
};
// tile_cfg: 0 = 16x8, 1 = 8x8, 2 = 16x16, 3 = 32x8 pixels per CTA.  pr: the
// run's distinct block records by value (at most kParamRecs; the views'
// lists in a.vidx), or null for records in a.recs (staged into shared memory).
void batch_tile_shape(int tile_cfg, int *tw, int *th);
cudaError_t launch_march_batch(const BatchArgs &a, int tile_cfg, int grid, cudaStream_t st,
                               const ParamRecs *pr = nullptr);

// K4 / K5: packing and occupancy (pack.cu)
cudaError_t launch_amax8(const float *x, int64_t n_vec, unsigned *amax_bits, cudaStream_t st);
// FP32 packs in the natural layout; FP16 / BF16 / FP8 in the pair layout
// (element i = vertex i and vertex i+1 of its row of `row` vertices).
cudaError_t launch_pack(const float *x, int64_t n_vec, int row, int dtype, const float *inv_scale8, void *out,
                        cudaStream_t st);
cudaError_t launch_occupancy(const float *grid, int R, int C, double log_thresh, uint32_t *bits, cudaStream_t st);
cudaError_t launch_pack_quad8(const float *x, int P, const float *inv_scale8, void *out, cudaStream_t st);
// Grid element layouts (k_pack_grid): one FP32 vertex; a vertex pair along x
// (FP16 / BF16 / FP8); a 2x2 quad of FP8 vertices over (x, y); the BF16
// channel 0 of a voxel's eight corners.
constexpr int kLayNat = 0, kLayPair = 1, kLayQuad8 = 2, kLayOct16 = 3;
// Pack a grid (R^3 x 8 FP32 master) into n_elem elements of `layout`, dense
// (blist null: element strides sy = R, sz = R^2) or brick-sparse (slot s of
// belem elements holds brick blist[s], nb bricks per axis, strides sy, sz
// inside a brick).  inv_scale8 may be null (scale 1).
cudaError_t launch_pack_grid(const float *x, int R, int64_t n_elem, int sy, int sz, int belem, const int32_t *blist,
                             int nb, int dtype, int layout, const float *inv_scale8, void *out, cudaStream_t st);

}  // namespace cow
