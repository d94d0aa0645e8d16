// cow_internal.h -- host-side context and helpers shared by the libcow
// translation units (not part of the C ABI).
#pragma once

#include <cmath>
#include <cstdarg>
#include <memory>
#include <string>
#include <vector>

#include <nvtx3/nvToolsExt.h>

#include "cow.h"
#include "cow_common.cuh"
#include "cow_kernels.h"

namespace cowi {

extern thread_local std::string g_last_error;

// Record a message for cow_last_error and return `st`.
cow_status fail(cow_status st, const char *fmt, ...);

bool is_device_ptr(const void *p);

#define COW_CUDA(call)                                                                      \
    do {                                                                                    \
        cudaError_t e_ = (call);                                                            \
        if (e_ != cudaSuccess) {                                                            \
            return cowi::fail(e_ == cudaErrorMemoryAllocation ? COW_ERR_OOM : COW_ERR_CUDA, \
                              "%s failed: %s", #call, cudaGetErrorString(e_));              \
        }                                                                                   \
    } while (0)

// An NVTX range around one C-ABI call (header-only NVTX v3: a no-op unless a
// profiler that collects NVTX, such as Nsight Systems or ncu with
// --nvtx, is attached).
struct NvtxRange {
    explicit NvtxRange(const char *name) { nvtxRangePushA(name); }
    ~NvtxRange() { nvtxRangePop(); }
    NvtxRange(const NvtxRange &) = delete;
    NvtxRange &operator=(const NvtxRange &) = delete;
};
#define COW_NVTX(name) cowi::NvtxRange cow_nvtx_range_(name)

// Restores the caller's current device when it leaves scope.
struct DeviceGuard {
    int prev = -1;
    explicit DeviceGuard(int dev) {
        if (cudaGetDevice(&prev) != cudaSuccess) prev = -1;
        if (prev != dev) cudaSetDevice(dev);
    }
    ~DeviceGuard() {
        int cur;
        if (prev >= 0 && cudaGetDevice(&cur) == cudaSuccess && cur != prev) cudaSetDevice(prev);
    }
};

// A device buffer that only grows.
struct DevBuf {
    void *p = nullptr;
    size_t cap = 0;
    cudaError_t reserve(size_t bytes) {
        if (bytes <= cap) return cudaSuccess;
        if (p) cudaFree(p);
        p = nullptr;
        cap = 0;
        cudaError_t e = cudaMalloc(&p, bytes);
        if (e == cudaSuccess) cap = bytes;
        return e;
    }
    void release() {
        if (p) cudaFree(p);
        p = nullptr;
        cap = 0;
    }
};

// A CUDA event owned by reference count: the calls that read a block record
// one after their kernels, and the block keeps the latest until it is
// unloaded (the unload waits for it).
struct SharedEvent {
    cudaEvent_t e = nullptr;
    SharedEvent() { cudaEventCreateWithFlags(&e, cudaEventDisableTiming); }
    ~SharedEvent() {
        if (e) cudaEventDestroy(e);
    }
    SharedEvent(const SharedEvent &) = delete;
    SharedEvent &operator=(const SharedEvent &) = delete;
};

struct BlockHost {
    float lo[3], hi[3];
    int32_t lod, parent, R, P;
    void *grid = nullptr;
    void *planes[3] = {nullptr, nullptr, nullptr};
    uint32_t *occ = nullptr;
    uint32_t *occ2 = nullptr;  // coarse occupancy level (OR over kOccGroup^3 cells)
    int64_t occ2_words = 0;
    // dynamic loading (cow_set_residency): the packed grid and planes may live
    // only in pinned host memory while the block is unloaded, as one buffer
    // (tensor t at feature_offset(t)); a loaded block's tensors are one chunk
    // of the context's stream-ordered pool at the same offsets
    void *host_feat = nullptr;
    void *chunk = nullptr;     // null while the tensors are the load-time allocations
    std::shared_ptr<SharedEvent> use_ev;  // after the last enqueued kernel that reads the block
    int32_t unb = 0;           // cow_set_block_unbounded flags
    bool resident = true;
    bool dirty = false;        // device copy newer than host_feat (cow_update_features)
    uint64_t last_use = 0;
    float *scale = nullptr;
    int32_t scale_exp[4][8];
    int64_t occ_words = 0;
    double ztop = 0.0;
    std::vector<int32_t> children;
    // brick-sparse grid (cow_load_blocks_ex with COW_LOAD_BRICKS): the stored
    // bricks, always resident like the occupancy levels
    int32_t Nb = 0;                 // bricks per axis; 0 = dense grid
    int32_t n_bricks = 0;           // stored bricks
    int32_t *brick_tab = nullptr;   // device, Nb^3: slot of each brick, -1 = not stored
    int32_t *brick_list = nullptr;  // device, n_bricks: brick id (bz Nb + by) Nb + bx of each slot
};

inline double focal_length(int32_t H, double fov_y_deg) {
    return (0.5 * (double)H) / tan(0.5 * fov_y_deg * M_PI / 180.0);
}

}  // namespace cowi

struct cow_ctx;
struct cow_batch;

namespace cowi {

// Device bytes of block i's packed features (what the residency budget counts).
int64_t block_feature_bytes(const cow_ctx *c, int32_t i);

// Make the blocks ids[0 .. n) resident under the context's budget (LRU
// unloading of the others); a no-op without a budget.  Block records of
// loaded or unloaded blocks are rewritten (cow_ctx::rec_gen advances); work
// enqueued on st afterwards waits for the loads.
cow_status make_resident(cow_ctx *c, const int32_t *ids, int64_t n, cudaStream_t st);

// Context internals for the scene files (scene_io.cu): packed bytes of
// tensor t of a block (0 grid with its density octets, 1-3 planes), its
// offset in a block's host copy, a block's kernel record, and teardown.
int64_t block_tensor_bytes(const cow_ctx *c, const BlockHost &b, int t);
int64_t block_feature_offset(const cow_ctx *c, const BlockHost &b, int t);
cow::BlockRec block_record(const cow_ctx *c, const BlockHost &b);
void destroy_context(cow_ctx *c);

// cow_free of a context with live batches: the batch drops its context
// pointer (its later calls fail with INVALID_ARG; cow_batch_free still works).
void batch_detach(struct cow_batch *b);

// After a call's kernels on st: under a budget, the blocks ids[0 .. n)
// remember that their next unload waits for this point of st.
cow_status note_use(cow_ctx *c, const int32_t *ids, int64_t n, cudaStream_t st);

}  // namespace cowi

struct cow_ctx {
    int device = 0;
    int dtype = 0;
    bool bricks = false;  // brick-sparse grids
    int occ_cell = 4;
    float occ_thresh = 0.01f;
    int schedule = COW_SCHED_THREAD_CONST;
    int tile_strip = 0;  // cow_set_tile_order
    uint32_t test_flags = 0, wait_polls = 0;  // cow_set_test_hooks
    std::vector<cowi::BlockHost> blocks;
    std::vector<cow::BlockRec> recs;  // block records (kernels receive copies by value)
    unsigned *d_err = nullptr;
    float *d_mlp = nullptr;
    cowi::DevBuf views, out_rgb, out_aux, out_nsamp;
    cowi::DevBuf gptrs, partials;  // backward: per-block gradient pointers, per-CTA MLP-gradient rows
    cowi::DevBuf f64ptrs;          // cow_render_rays_f64: per-block FP64 feature pointers
    cowi::DevBuf staging;          // host masters of cow_update_features
    cowi::DevBuf block_mlps;       // cow_set_block_mlps: n_blocks x block_mlp_nparam FP32
    cowi::DevBuf bm_scratch;       // backward of the per-block MLP form: 2 x n_rays x n_ids x 8 FP32
    int ray_order = COW_RAY_ORDER_COHERENT;  // cow_set_ray_order
    cowi::DevBuf ray_keys, ray_hist, ray_perm;  // the coherent order of the last ray-batch call
    int32_t n_freq = -1;           // PE frequencies of block_mlps; -1 = none set
    int32_t block_mlp_nparam = 0;
    // dynamic loading: budget for the packed features on the device (0 = all
    // resident), LRU clock and counters
    int64_t budget = 0;
    uint64_t use_clock = 0;
    int64_t resident_bytes = 0;
    int64_t n_uploads = 0, upload_bytes = 0, n_evictions = 0;
    int64_t n_evict_wait_last = 0;              // unloads behind the kernels of the call just before
    std::shared_ptr<cowi::SharedEvent> last_call_ev;  // the use event of the most recent call
    std::vector<struct cow_batch *> batches;  // live cow_batch objects on this context (cow_free detaches them)
    uint64_t rec_gen = 0;   // advances whenever a block record is rewritten
    cudaMemPool_t pool = nullptr;  // loads under a budget allocate from it (created with the first budget)
    // loads and unloads run on their own stream, ordered by events: an unload
    // waits for the kernels that read the block, a call's kernels wait for
    // the loads it needs, so a call's loads can overlap earlier calls' kernels
    cudaStream_t copy_stream = nullptr;
    cudaEvent_t loaded = nullptr;  // recorded on copy_stream after a call's loads
};

namespace cowi {

// The DT a context's kernels are instantiated for: the storage dtype, with
// cow::kBrickBit for brick-sparse grids.
inline int kernel_dtype(const cow_ctx *c) { return c->dtype | (c->bricks ? cow::kBrickBit : 0); }

}  // namespace cowi
