/*
 * cow.h -- C ABI of libcow: block-based volume rendering of baked MERF-style
 * scene blocks on one NVIDIA GB300 (sm_103a), after City-on-Web
 * (arXiv 2312.16457).
 *
 * The problem the calls solve (Sec. 4.1 rendering stage, Sec. 4.2, App. D):
 * given a scene partitioned on the ground plane into blocks, each baked at
 * several levels of detail into a low-resolution 3D feature grid plus three
 * high-resolution feature planes, and given cameras, render images with
 * correct occlusion between blocks: per pixel, march the ray through every
 * selected block (Eq. 1-2 within a block, Eq. 11), composite the blocks in
 * depth order (Eq. 5 / Eq. 12) and shade the composited diffuse colour and
 * specular feature with one deferred MLP (Eq. 3).
 *
 * Conventions for every call:
 *  - No C++ exception crosses this boundary.  Every call returns a
 *    cow_status; on failure cow_last_error() returns a message (thread-local,
 *    valid until the next call on the same thread).
 *  - Caller-owned inputs are read-only and may be freed when the call
 *    returns.  A context owns its packed device copies until cow_free.
 *  - Outputs are caller-allocated.  Device work is enqueued asynchronously on
 *    the caller's CUDA stream (`stream` is a cudaStream_t; NULL = legacy
 *    default stream).  Calls that use one context must be issued on one stream
 *    or be ordered by the caller, because a context reuses its per-call
 *    device buffers.
 *  - Kernels that detect a fault (a sample range beyond the bound, a wait
 *    that ran out) set an error word instead of trapping; cow_sync_check
 *    reports it as COW_ERR_DEVICE_ASSERT or COW_ERR_TIMEOUT.
 *
 * Notation: block b has the world AABB [lo, hi]; R = grid vertices per axis,
 * P = plane texels per axis.  Channels: 0 pre-activation log-density
 * (sigma = exp), 1-3 diffuse colour, 4-7 specular feature (sigmoid).
 */
#ifndef COW_H
#define COW_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define COW_NCH 8           /* feature channels per grid vertex / plane texel */
#define COW_MLP_NPARAM 499  /* deferred MLP 10 -> 16 -> 16 -> 3 */

typedef enum cow_status {
    COW_OK = 0,
    COW_ERR_INVALID_ARG = 1,   /* a null pointer, size or layout the call rejects */
    COW_ERR_CUDA = 2,          /* a CUDA runtime call failed (message has the CUDA error) */
    COW_ERR_OOM = 3,           /* device allocation failed */
    COW_ERR_UNSUPPORTED = 4,   /* valid request this build does not implement */
    COW_ERR_TIMEOUT = 5,       /* a bounded device-side wait ran out */
    COW_ERR_DEVICE_ASSERT = 6  /* a kernel's own range check fired */
} cow_status;

/* Storage format of the packed features (Sec. 4.5 bakes 8-bit textures; the
 * formats here are the GPU equivalents).  FP8 uses per-channel power-of-two
 * scales: channel c of each tensor is stored as x / 2^e_c with the smallest
 * e_c such that max|x_c| <= 448 * 2^e_c.  FP32 / FP16 / BF16 use scale 1.
 * Conversion is round-to-nearest-even (FP8 saturating at +-448). */
/* Storage of the packed features (the math is FP32 in every case).
 * COW_BF16_FP8: the grid in BF16 and the three planes in FP8-E4M3 with
 * per-channel power-of-two scales, the planes in a quad layout (one 32-byte
 * element holds the 2x2 texels of a bilinear footprint), so a sample takes 7
 * gathers instead of 10.
 * COW_FP8_BF16D: FP8-E4M3 features with per-channel power-of-two scales,
 * except the grid's channel 0 (log-density), which is kept in BF16 (no
 * scale): E4M3's 3-bit mantissa on a log-density near 3 moves sigma by up to
 * 13 %, more than the precision form's 1e-2 colour bound allows, while the
 * colour and specular channels and the planes' small values keep it.  The
 * grid and planes are stored in the quad layout (2 x 2 FP8 vertices or texels
 * in 32 bytes) and the density as the eight corners of each voxel (16
 * bytes), so a sample takes 6 gathers (176 bytes). */
typedef enum cow_dtype {
    COW_FP32 = 0,
    COW_FP16 = 1,
    COW_BF16 = 2,
    COW_FP8_E4M3 = 3,
    COW_BF16_FP8 = 4,
    COW_FP8_BF16D = 5
} cow_dtype;

/* One baked block at one level of detail (Sec. 4.1: f^{k,l}; LOD l merges 2x2
 * blocks of level l-1, Sec. 4.1 and Sec. 4.4). */
typedef struct cow_block_desc {
    float lo[3], hi[3];      /* world AABB; xy footprints of one level tile the ground */
    int32_t lod;             /* level of detail, 1 = finest */
    int32_t parent;          /* index (in this array) of the covering block one level up, -1 if none */
    int32_t grid_res;        /* R >= 2; vertex 0 at lo, vertex R-1 at hi (vertex-aligned) */
    int32_t plane_res;       /* P >= 2; sample spacing delta = (hi_x - lo_x) / P */
    const float *grid;       /* FP32 master, R^3 x 8, index ((z*R + y)*R + x)*8 + c; host or device */
    const float *planes[3];  /* FP32 master, P^2 x 8 each, index (v*P + u)*8 + c; planes xy, xz, yz */
} cow_block_desc;

/* Pinhole camera: 3x4 row-major camera-to-world matrix with OpenGL axes
 * (the camera looks along -z, +y up), image size and vertical field of view.
 * Pixel (x, y) shoots the ray through its centre (x + 1/2, y + 1/2). */
typedef struct cow_camera {
    double c2w[12];
    int32_t width, height;
    double fov_y_deg;
} cow_camera;

typedef struct cow_ctx cow_ctx;

/* render flags */
#define COW_FLAG_MLP_BF16 1u    /* deferred MLP with BF16 operands and FP32 accumulation */
#define COW_FLAG_BLOCK_MLPS 2u  /* per-block deferred MLPs blended by Eq. 5 (cow_set_block_mlps) */

/* Upload and pack a set of blocks (all levels) on the current CUDA device.
 *   out        : receives the new context (owned by the caller; cow_free).
 *   blocks, n  : n >= 1 descriptors; arrays may be host or device memory.
 *   storage    : packed format of the grid and planes.
 *   occ_thresh : occupancy threshold on density (Sec. 4.5 bakes a binary
 *                occupancy grid; here a cell is occupied when any grid vertex
 *                of it has exp(ch0) > occ_thresh, decided on the FP32 master
 *                as (double)ch0 > log((double)occ_thresh)).
 *   occ_cell   : voxels per occupancy-cell edge (1..4096); a block has
 *                ceil((R-1)/occ_cell)^3 cells; cell c spans vertices
 *                [c*occ_cell, c*occ_cell + occ_cell] along each axis.
 *   stream     : packing kernels run on it; the call synchronises it before
 *                returning, so the masters may be freed afterwards.
 * Errors: INVALID_ARG (null pointer, R or P < 2, lo >= hi, bad dtype),
 * OOM, CUDA. */
cow_status cow_load_blocks(cow_ctx **out, const cow_block_desc *blocks, int32_t n, cow_dtype storage,
                           float occ_thresh, int32_t occ_cell, void *stream);

/* Load flags of cow_load_blocks_ex. */
#define COW_LOAD_BRICKS 1u /* brick-sparse grids (below) */

/* cow_load_blocks with load flags (0 = cow_load_blocks).
 * COW_LOAD_BRICKS stores every grid brick-sparse, the GPU form of the sparse
 * voxel grid behind an indirection table that the paper's baked blocks use
 * (Sec. 3 on MERF / SNeRG-style representations, Sec. 4.5 baking): the grid
 * is cut into bricks of 16 voxels per edge (one coarse occupancy cell, 4 x 4 x
 * 4 cells of occ_cell = 4 voxels); only bricks with an occupied cell are
 * stored, each with the grid elements of its voxels (a halo of one vertex on
 * the far faces), and a per-block table of ceil((R-1)/16)^3 int32 slots
 * (-1 = empty brick) maps a voxel to its brick.  Lattice samples lie in
 * occupied cells, whose bricks are stored, so renders, ray batches and
 * gradients equal those of the dense grid bit for bit.  Device memory is the
 * stored bricks (about 1.13x their voxels in the pair layout) plus the table.
 * Errors as cow_load_blocks; UNSUPPORTED for occ_cell != 4.  On a
 * brick-sparse context cow_sparsity_loss (it samples arbitrary points) and
 * cow_export_packed of the grid return UNSUPPORTED. */
cow_status cow_load_blocks_ex(cow_ctx **out, const cow_block_desc *blocks, int32_t n, cow_dtype storage,
                              float occ_thresh, int32_t occ_cell, uint32_t load_flags, void *stream);

/* Packed scene files (the paper bakes its blocks to texture assets, Sec.
 * 4.5; this is the GPU equivalent, no counterpart of the format in the
 * paper): cow_save_scene writes what a context holds -- every block's packed
 * features in the storage format (dense or brick-sparse), occupancy levels,
 * FP8 scales, z_top and LOD links -- as a binary header and block table, a
 * JSON manifest of the same facts, then the raw arrays (unloaded blocks are
 * written from their host copies).  cow_load_scene creates a context from
 * such a file on the current device with every block resident, without the
 * FP32 masters or a re-pack; its renders equal the saved context's bit for
 * bit.  Errors: INVALID_ARG (unreadable, truncated or foreign file, write
 * failure), OOM, CUDA. */
cow_status cow_save_scene(const cow_ctx *ctx, const char *path);
cow_status cow_load_scene(cow_ctx **out, const char *path, void *stream);

/* Release a context and all its device memory (NULL is accepted). */
cow_status cow_free(cow_ctx *ctx);

/* Number of blocks held, and the z of the highest occupied part of block i
 * (App. D: the top of its highest occupied cell row, lo_z if empty). */
cow_status cow_num_blocks(const cow_ctx *ctx, int32_t *out_n);
cow_status cow_block_ztop(const cow_ctx *ctx, int32_t block, double *out_ztop);

/* LOD selection, visibility and depth sort of the real-time viewer (App. D),
 * on the host in FP64.
 *   A block is visible unless all 8 corners of [lo_x,hi_x] x [lo_y,hi_y] x
 *   [lo_z, ztop] lie strictly outside one of the five planes of the view
 *   pyramid.  Starting from the visible blocks of the coarsest level, a
 *   block of level l > 1 is selected when every visible child is farther than
 *   lod_thresh[l-2] from the camera (distance to (centre_x, centre_y, ztop));
 *   otherwise its visible children are examined.  Level-1 blocks are always
 *   selected.  The result is sorted near to far by the xy distance of block
 *   centres to the camera (ties by index).
 *   lod_thresh : n_lod thresholds; lod_thresh[k] applies to level k+1.
 *   out_ids    : host array of cap entries; out_n receives the count (if it
 *                exceeds cap, nothing is written and INVALID_ARG is returned). */
cow_status cow_select_lod(const cow_ctx *ctx, const cow_camera *cam, const double *lod_thresh, int32_t n_lod,
                          int32_t *out_ids, int32_t cap, int32_t *out_n);

/* Depth sort only (App. D): ids sorted near to far by the xy distance of
 * block centres to the camera, ties by index.  Host arrays of n entries. */
cow_status cow_sort_blocks(const cow_ctx *ctx, const cow_camera *cam, const int32_t *ids, int32_t n, int32_t *out);

/* Render n_views images (Eq. 1-2, 5/12 and 3).
 *   cams        : host array of n_views cameras.
 *   ids         : host array, the block ids of view v (near to far, e.g. from
 *                 cow_select_lod) are ids[ids_offsets[v] .. ids_offsets[v+1]).
 *   mlp         : 499 FP32 deferred-MLP parameters W1[10][16], b1[16],
 *                 W2[16][16], b2[16], W3[16][3], b3[3] (input-major); the
 *                 MLP input is [C_d (3), F (4), d (3)]; C = C_d + sigmoid(...).
 *                 Host or device.
 *   ert_eps     : a ray stops once its transmittance falls below ert_eps
 *                 (0 = never); the colour changes by at most ert_eps per
 *                 channel of C_d and F.
 *   flags       : 0, COW_FLAG_MLP_BF16, or COW_FLAG_BLOCK_MLPS: every block
 *                 k then computes its own colour C^k = C_d^k + Phi^k(C_d^k,
 *                 F^k, PE(d)) with the MLP set by cow_set_block_mlps, and the
 *                 block colours are blended near to far by Eq. 5,
 *                 C = sum_k prod_{j<k} (1 - alpha^j) C^k, over the blocks in
 *                 which the ray has at least one occupied sample; `mlp` is
 *                 not read (may be NULL).  Runs the thread schedule (records
 *                 in the parameter buffer when they fit, as
 *                 COW_SCHED_THREAD_CONST); FP32 MLP math only (INVALID_ARG
 *                 together with COW_FLAG_MLP_BF16, or when no block MLPs
 *                 are set).  cow_render_rays, cow_render_backward and the
 *                 batched form take neither this flag nor the per-block MLPs.
 *   out_rgb     : float32, (sum of W*H) x 3, views in order, rows top to
 *                 bottom.  Device memory, or host memory: page-locked memory
 *                 mapped into the device's address space (cudaHostAlloc on
 *                 a system with unified addressing) is written by the kernel
 *                 directly; other host memory is rendered into context
 *                 buffers and copied.  Host outputs are complete when the
 *                 stream completes (pageable ones when the call returns).
 *   out_aux     : NULL or float32 (sum W*H) x 8: C_d (3), F (4) and the
 *                 transmittance left after the last block; same rules.
 *   out_nsamp   : NULL or int32 (sum W*H): occupied samples marched per pixel.
 * Errors: INVALID_ARG (bad id, size, pointer), OOM, CUDA. */
cow_status cow_render(cow_ctx *ctx, const cow_camera *cams, int32_t n_views, const int32_t *ids,
                      const int32_t *ids_offsets, const float *mlp, float ert_eps, uint32_t flags, float *out_rgb,
                      float *out_aux, int32_t *out_nsamp, void *stream);

/* Unbounded boundary blocks (implementation details of the paper: blocks on
 * the scene's boundary use MERF's scene contraction, Eq. 16).  A contracted
 * block's grid and planes span u = contract(x) in [-2, 2]^3, x = (p - c) / h
 * with c the centre and h the half extents of its box: contract(x) = x
 * inside the unit cube; outside, 2 - 1/|x_j| (sign of x_j) on the
 * coordinates that reach ||x||_inf and x_j / ||x||_inf on the others.  The
 * block owns its xy footprint extended to infinity across the flagged sides
 * (half-open as Eq. 4) and every z.  A ray marches it from its first owned
 * lattice point (t = (i + 1/2) delta) with steps s = delta m^2,
 * m = max(1, ||x||_inf), until it leaves the region, ||x||_inf > 1e4 or 65536
 * steps; a sample's alpha is 1 - exp(-sigma s).
 *   flags : 0 (bounded, the default) or COW_UNBOUNDED_CONTRACTED | sides.
 * The grid and planes given at load time are read in u (vertex 0 at u = -2,
 * vertex R-1 at u = 2); occupancy is built from them as for any block.
 * Errors: INVALID_ARG. */
#define COW_UNBOUNDED_XLO 1
#define COW_UNBOUNDED_XHI 2
#define COW_UNBOUNDED_YLO 4
#define COW_UNBOUNDED_YHI 8
#define COW_UNBOUNDED_CONTRACTED 16
cow_status cow_set_block_unbounded(cow_ctx *ctx, int32_t block, int32_t flags, void *stream);

/* Per-block deferred MLPs (Sec. 4.1: each block k of LOD l carries its own
 * tiny MLP Phi^{k,l}; Sec. 4.2, Eq. 5: the block colours of Eq. 3 are
 * blended by opacity) with a multi-frequency encoding of the view direction.
 *   mlps   : n_mlps x nparam FP32, row i for block i of the context (all
 *            levels, in load order), host or device; copied into the
 *            context.  NULL with n_mlps = 0 removes them.  Each row is
 *            W1[n_in][16], b1[16], W2[16][16], b2[16], W3[16][3], b3[3]
 *            (input-major), n_in = 10 + 6 n_freq, nparam = 16 n_in + 339.
 *            The input is [C_d^k (3), F^k (4), PE(d)] with
 *            PE(d) = d, then for l = 0 .. n_freq-1 sin(2^l d) (x, y, z) and
 *            cos(2^l d) (x, y, z).
 *   n_freq : 0 .. 8.
 * Errors: INVALID_ARG (n_mlps other than the context's block count, n_freq
 * out of range, NULL pointer), OOM, CUDA.  The copy is ordered on `stream`:
 * a render still running on another stream must be finished first. */
cow_status cow_set_block_mlps(cow_ctx *ctx, const float *mlps, int32_t n_mlps, int32_t n_freq, void *stream);

/* Dynamic loading and unloading under a device-memory budget (App. D's
 * dynamic loading strategy; Sec. 1 lists it with LOD as the way resources are
 * managed).  A block's loadable resources are its packed grid and planes
 * (cow_block_bytes); occupancy, scales and records stay resident.
 *   cow_set_residency : budget_bytes > 0 keeps a pinned host copy of every
 *       block's packed features and unloads every block from the device;
 *       from then on each cow_render / cow_render_rays / cow_render_backward
 *       / cow_update_features call loads the blocks it uses, after unloading
 *       the least recently used blocks it does not use (ties: lowest index)
 *       until they fit.  A call whose blocks alone exceed the budget fails
 *       with COW_ERR_OOM and changes nothing.  Setting a smaller budget
 *       unloads least recently used blocks; 0 loads every block back and
 *       frees the host copies.  Features changed by cow_update_features are
 *       copied back to the host copy before their block is unloaded.
 *       Loads and unloads are ordered on the calling stream and the call
 *       returns without waiting for them (a context serves one stream at a
 *       time in this mode); the host waits only to copy changed features
 *       back and to free the allocations made when the blocks were loaded.  The batched form serves its views in runs whose blocks
 *       fit the budget together (cow_batch_render); cow_render_backward_noalloc
 *       loads nothing and rejects unloaded blocks (INVALID_ARG).
 *   cow_get_residency : the budget, the bytes and blocks now on the device
 *       and the load / unload counters since the context was created.
 *   cow_block_bytes   : bytes of block's packed grid and planes on the device. */
typedef struct {
    int64_t budget_bytes;
    int64_t resident_bytes;
    int32_t resident_blocks;
    int64_t uploads;       /* blocks loaded */
    int64_t upload_bytes;  /* bytes copied host -> device by loads */
    int64_t evictions;     /* blocks unloaded */
    int64_t evictions_waiting_last_call; /* unloads that had to wait for the kernels of the call just
                                            before (a load behind them cannot overlap that call) */
} cow_residency;
cow_status cow_set_residency(cow_ctx *ctx, int64_t budget_bytes, void *stream);
cow_status cow_get_residency(const cow_ctx *ctx, cow_residency *out);
cow_status cow_block_bytes(const cow_ctx *ctx, int32_t block, int64_t *out_bytes);

/* Residency-aware order of views (host only, needs no context or GPU): given
 * each block's bytes and every view's block ids (CSR, as cow_render), pick an
 * order that loads few bytes under budget_bytes, greedily taking next the
 * view that loads the fewest bytes given what the previous views left
 * resident.  It simulates exactly the loading rule of cow_set_residency
 * (from its cold start, one view per call), so rendering the views one per
 * cow_render call in out_order loads *out_upload_bytes bytes;
 * *out_upload_bytes_given (may be NULL) is the same for the given order.
 *   out_order : n_views view indices.
 * Errors: INVALID_ARG (bad sizes or ids, a view needing more than the budget). */
cow_status cow_plan_view_order(const int64_t *block_bytes, int32_t n_blocks, const int32_t *ids,
                               const int32_t *ids_offsets, int32_t n_views, int64_t budget_bytes, int32_t *out_order,
                               int64_t *out_upload_bytes, int64_t *out_upload_bytes_given);

/* Improve a view order (host only): starting from io_order (a permutation
 * of 0 .. n_views-1, for example cow_plan_view_order's), move one view at a
 * time to another place and keep a move when the same simulation of the
 * loading rule loads fewer bytes; rescan after each kept move and stop when
 * no move helps or after max_evals simulated orders (deterministic).
 * io_order receives the result, *out_upload_bytes (may be NULL) its bytes,
 * never more than the input order's.  Each evaluation costs one simulation
 * (about n_views x n_blocks steps).
 * Errors: INVALID_ARG (as cow_plan_view_order, io_order not a permutation,
 * max_evals < 1). */
cow_status cow_refine_view_order(const int64_t *block_bytes, int32_t n_blocks, const int32_t *ids,
                                 const int32_t *ids_offsets, int32_t n_views, int64_t budget_bytes, int32_t *io_order,
                                 int32_t max_evals, int64_t *out_upload_bytes);

/* Batched form: many cameras of uneven size and LOD set served by
 * persistent launches over a (view, tile, block) work queue.  Every CTA takes
 * the next (view, tile) item from a device counter, culls the view's block
 * list against the tile's pyramid (blocks that no ray of the tile can sample)
 * and marches the tile's rays; each pixel equals cow_render's bit for bit.
 * When every view has at most 96 blocks the views are grouped into runs
 * whose distinct blocks fit one launch's parameter buffer (96 records, read
 * through the constant cache), one persistent launch a run; otherwise one
 * launch stages each view's records into shared memory.  The launches can
 * be replayed from one CUDA graph, and their tile shape and resident CTAs
 * per SM can be picked by cow_batch_tune, which times the candidates on the
 * batch that is set.
 *
 * cow_batch_create : pinned + device staging for up to max_views cameras and
 *                    max_ids block ids (sum over views); owned by the caller
 *                    (cow_batch_free before the context).
 * cow_batch_set_views : the cameras and their near-to-far block ids (CSR, as
 *                    cow_render); out_pixels (may be NULL) receives the total
 *                    pixel count, the rows of the outputs.  Waits for the
 *                    previous batch's staging copy before rewriting it.
 * cow_batch_render : outputs as cow_render but device memory only; use_graph
 *                    != 0 replays a CUDA graph captured on the first call (and
 *                    again whenever the arguments or the configuration change).
 *                    Under a residency budget (cow_set_residency) the views
 *                    are cut, in the order set, into runs: a view joins the
 *                    current run while the run's distinct blocks plus its own
 *                    fit the run fraction of the budget (1/2 by default, so
 *                    a run's loads overlap the previous run's marching; a
 *                    view above it forms its own run), else it starts the
 *                    next run.  Successive
 *                    renders walk the views first to last, then last to
 *                    first, and so on (cow_batch_set_views restarts at first
 *                    to last), so each render begins with the blocks the
 *                    previous one left resident.  Each run's
 *                    blocks are made resident by the cow_render rule (LRU
 *                    unloading of the others) and the run is one persistent
 *                    launch; use_graph is then ignored.  Pixels equal the all-resident
 *                    batch's.  A view whose own blocks exceed the budget
 *                    fails with OOM (runs cut before it may have rendered).
 *                    cow_plan_view_order gives an order that loads few bytes.
 * cow_batch_last_groups : launches (runs) of the last cow_batch_render.
 * cow_batch_set_config : tile_cfg 0 = 16x8, 1 = 8x8, 2 = 16x16, 3 = 32x8
 *                    pixels per CTA; 4 = warp items, 8x4 pixels per warp,
 *                    each warp taking its own items (no CTA barrier in the
 *                    loop; records in the parameter buffer only, else
 *                    cow_batch_render fails with UNSUPPORTED); ctas_per_sm
 *                    resident CTAs per SM (1..32).
 * cow_batch_tune   : times every (tile_cfg, ctas_per_sm in {2,3,4,6,8}) on the
 *                    set views (reps renders each, into out_rgb) with the
 *                    records in the parameter buffer, then the best of them
 *                    with the records staged in shared memory, then (without
 *                    a residency budget) the grid schedule, and keeps the
 *                    fastest; reports the queue's best tile and CTAs and the
 *                    kept time per batch in ms (cow_batch_get_config: the
 *                    record mode; cow_batch_get_schedule: the schedule).
 * Errors: INVALID_ARG, OOM, CUDA. */
typedef struct cow_batch cow_batch;
cow_status cow_batch_create(cow_ctx *ctx, int32_t max_views, int32_t max_ids, cow_batch **out);
cow_status cow_batch_free(cow_batch *b);
cow_status cow_batch_set_views(cow_batch *b, const cow_camera *cams, int32_t n_views, const int32_t *ids,
                               const int32_t *ids_offsets, int64_t *out_pixels);
cow_status cow_batch_render(cow_batch *b, const float *mlp, float ert_eps, uint32_t flags, float *out_rgb,
                            float *out_aux, int32_t *out_nsamp, int32_t use_graph, void *stream);
cow_status cow_batch_last_groups(const cow_batch *b, int32_t *out_groups);
/* The fraction of the residency budget one run of cow_batch_render may fill
 * (0 < frac <= 1; default 0.5).  Errors: INVALID_ARG. */
cow_status cow_batch_set_run_fraction(cow_batch *b, float frac);
/* Where the batched kernels read block records (the batch's marching
 * schedule): COW_BATCH_RECORDS_PARAM (default) groups the views into runs
 * whose records travel in the launch's parameter buffer (when every view has
 * at most 96 blocks, else as SHARED); COW_BATCH_RECORDS_SHARED has one launch
 * stage each view's records into shared memory.  cow_batch_tune picks it
 * (after tile shape and CTAs per SM); cow_batch_get_config reports the
 * configuration in use.  Errors: INVALID_ARG. */
#define COW_BATCH_RECORDS_PARAM 0
#define COW_BATCH_RECORDS_SHARED 1
cow_status cow_batch_set_records(cow_batch *b, int32_t mode);
/* How cow_batch_render schedules the views' tiles without a residency
 * budget: COW_BATCH_SCHED_QUEUE (default), the persistent launches over the
 * (view, tile) work queue described above; COW_BATCH_SCHED_GRID, the view
 * marcher of cow_render -- one CTA per 16x8 tile, scheduled by the
 * hardware -- on groups of consecutive views whose block lists, concatenated,
 * fit one launch's parameter buffer (96 records; a longer list forms its own
 * group), one launch per group, use_graph ignored.  The queue pays per tile
 * for its work counter and cull and gains on many small views; the grid
 * pays per launch.  Pixels are the same either way.  cow_batch_tune times
 * both.  Under a budget the queue is used.  Errors: INVALID_ARG. */
#define COW_BATCH_SCHED_QUEUE 0
#define COW_BATCH_SCHED_GRID 1
cow_status cow_batch_set_schedule(cow_batch *b, int32_t sched);
cow_status cow_batch_get_schedule(const cow_batch *b, int32_t *out_sched);
cow_status cow_batch_get_config(const cow_batch *b, int32_t *out_tile_cfg, int32_t *out_ctas_per_sm,
                                int32_t *out_records);
cow_status cow_batch_set_config(cow_batch *b, int32_t tile_cfg, int32_t ctas_per_sm);
cow_status cow_batch_tune(cow_batch *b, const float *mlp, float ert_eps, uint32_t flags, float *out_rgb, int32_t reps,
                          void *stream, int32_t *out_tile_cfg, int32_t *out_ctas_per_sm, float *out_ms);

/* Render independent rays (Sec. 4.2 training-stage form: each ray composites
 * the given blocks in the xy-distance order of its own origin, App. D).
 *   o, d        : device float32 n_rays x 3 origins and unit directions.
 *   ids, n_ids  : host array of the blocks to composite (1..64).
 *   other arguments as cow_render; outputs have n_rays rows.
 *   flags       : as cow_render; with COW_FLAG_BLOCK_MLPS each ray blends
 *                 its blocks by Eq. 5 with their own MLPs (cow_set_block_mlps)
 *                 and mlp may be NULL.  The gradient calls take the global
 *                 form only.
 * n_rays = 0 returns COW_OK at once (the arrays may then be NULL); the same
 * holds for cow_render_rays_block_t, cow_render_backward(_noalloc),
 * cow_opacity_loss and, with n_points = 0, cow_sparsity_loss. */
cow_status cow_render_rays(cow_ctx *ctx, const float *o, const float *d, int64_t n_rays, const int32_t *ids,
                           int32_t n_ids, const float *mlp, float ert_eps, uint32_t flags, float *out_rgb,
                           float *out_aux, int32_t *out_nsamp, void *stream);

/* Check aid for the differentiation form (FP64 on the GPU serves only the
 * finite-difference gradient check): the ray-batch render of
 * cow_render_rays without early termination, taking the same lattice samples
 * (decided by the FP32 sequence of the marcher) but computing every lookup
 * (Sec. 4.1 f^{k,l}), activation, weight (Eq. 1-2), composite (Eq. 12) and
 * the deferred MLP (Eq. 3) in FP64 from FP64 copies of the features:
 * grids[i] (R^3 x 8) and planes[3 i + k] (P^2 x 8) of block i, host arrays
 * of n_blocks / 3 n_blocks device pointers (only the blocks of ids are read;
 * the occupancy is the context's).  mlp: 499 FP64; out_rgb n x 3, out_aux n x
 * 8 (C_d, F, T; may be NULL), FP64 device memory.  A central difference of
 * it checks cow_render_backward at 1e-3 entry by entry.  Synchronises
 * stream.  Errors: INVALID_ARG, CUDA. */
cow_status cow_render_rays_f64(cow_ctx *ctx, const float *o, const float *d, int64_t n_rays, const int32_t *ids,
                               int32_t n_ids, const double *mlp, const double *const *grids,
                               const double *const *planes, double *out_rgb, double *out_aux, void *stream);

/* Block-parallel form of the ray-batch render (Sec. 4.2, Eq. 11-13; the
 * paper renders every block in its own shader and alpha-blends the images,
 * Sec. 4.2 and App. A).  Two calls:
 *   cow_render_partials: every block of ids marched alone, from an in-block
 *     transmittance of 1, for every ray: out_partials[(r * n_ids + k) * 8 ..]
 *     = (C_d^k (3), F^k (4), T^k) of block ids[k] (Eq. 11; T^k = 1 - alpha^k,
 *     = 1 with C_d^k = F^k = 0 for a ray that takes no sample in it).  No
 *     early termination.  The blocks may be split between calls or devices;
 *     each partial depends on its block alone.
 *   cow_composite_over (K2): per ray, the partials of ids folded near to far
 *     (App. D order from the ray's origin, as cow_render_rays) with the
 *     associative "over" of Eq. 12-13, (C, F, T) <- (C + T C^k, F + T F^k,
 *     T T^k), then the deferred MLP (Eq. 3): out_rgb (n x 3), out_aux (n x 8:
 *     C_d, F, T; may be NULL).  flags: 0 or COW_FLAG_MLP_BF16.
 * Composited partials equal cow_render_rays without early termination up to
 * FP32 rounding (the fused marcher carries T through the samples instead).
 * Arrays are device memory; partials 16-byte aligned.  Errors: INVALID_ARG,
 * OOM (residency budget), CUDA. */
cow_status cow_render_partials(cow_ctx *ctx, const float *o, const float *d, int64_t n_rays, const int32_t *ids,
                               int32_t n_ids, float *out_partials, void *stream);
cow_status cow_composite_over(cow_ctx *ctx, const float *o, const float *d, int64_t n_rays, const int32_t *ids,
                              int32_t n_ids, const float *partials, const float *mlp, uint32_t flags, float *out_rgb,
                              float *out_aux, void *stream);

/* cow_render_rays without early termination that also writes every block's
 * own transmittance prod (1 - alpha_i) over its occupied samples (Eq. 11),
 * -1 for a block without one: out_block_T is device float32 n_rays x n_ids,
 * row r, column k for ids[k].  cow_opacity_loss reads it instead of marching
 * each block a second time. */
cow_status cow_render_rays_block_t(cow_ctx *ctx, const float *o, const float *d, int64_t n_rays, const int32_t *ids,
                                   int32_t n_ids, const float *mlp, uint32_t flags, float *out_rgb, float *out_aux,
                                   int32_t *out_nsamp, float *out_block_T, void *stream);

/* Gradients of the ray-batch render (differentiation form): the analytic
 * adjoint of cow_render_rays with respect to every grid and plane feature and
 * every deferred-MLP parameter, given dL/dC per ray.  Each ray is marched
 * again over exactly the forward's samples (occupancy held fixed); the
 * contribution of the samples behind a sample is the forward's saved total
 * (out_aux) minus the running prefix, so nothing per sample is stored.
 *   o, d, ids, n_ids, mlp, ert_eps : as the forward call (device o, d, mlp);
 *   aux       : the forward's out_aux (device, n_rays x 8, 16-byte aligned);
 *   dL_drgb   : device float32 n_rays x 3;
 *   grad_grid : host array of n_blocks device pointers, R^3 x 8 FP32 each in
 *               the natural layout (NULL entries: no gradient for that block);
 *   grad_planes : host array of 3 x n_blocks device pointers, P^2 x 8 FP32;
 *   grad_mlp  : device float32 499.
 * All gradients are ACCUMULATED (+=); the caller zeroes them.  Gradients are
 * with respect to the feature values the lookup reads (the dequantised
 * values for FP16 / BF16 / FP8 storage).  Feature gradients use float
 * atomics (summation order varies between runs); the MLP gradient is summed
 * in a fixed order through per-CTA rows the context allocates.
 * Errors: INVALID_ARG, OOM, CUDA. */
cow_status cow_render_backward(cow_ctx *ctx, const float *o, const float *d, int64_t n_rays, const int32_t *ids,
                               int32_t n_ids, const float *mlp, float ert_eps, const float *aux, const float *dL_drgb,
                               float *const *grad_grid, float *const *grad_planes, float *grad_mlp, void *stream);

/* Allocation-free variant of cow_render_backward (the paper has no
 * counterpart; it exists for callers of this library that cannot allocate
 * device memory once running -- a trainer or viewer inside a fixed
 * device-memory budget, or a steady-state loop that must not pay for
 * cudaMalloc / cudaFree and the device synchronisation cudaFree implies).
 * Same arguments and results as cow_render_backward, with these differences:
 *  - no device or host allocation: the scratch (per-CTA MLP-gradient rows,
 *    per-ray dL/dC_d and dL/dF, the per-block gradient pointer table) lives
 *    in one static device array of the library (3 MiB, held by every GPU
 *    that loads the library until the process exits); the pointer table is
 *    written by a small kernel that takes the call's gradient pointers as
 *    launch parameters, so no enqueued work reads host memory after the
 *    call returns;
 *  - at most 65536 rays and 1024 context blocks per call; larger requests
 *    return COW_ERR_INVALID_ARG with a message naming the limit;
 *  - it loads no blocks: under a residency budget (cow_set_residency) a
 *    block of `ids` that is not on the device returns COW_ERR_INVALID_ARG
 *    (render the rays first), and the call does not refresh the blocks'
 *    least-recently-used order;
 *  - the first call on a device looks the array's device address up
 *    (cudaGetSymbolAddress); make that first call before any stream capture;
 *  - every call on a device shares the array and rewrites what it reads, so
 *    calls that overlap on the GPU (other streams, other contexts on the same
 *    device) race on it: order them.
 * Errors: INVALID_ARG, UNSUPPORTED (device index >= 64), CUDA. */
cow_status cow_render_backward_noalloc(cow_ctx *ctx, const float *o, const float *d, int64_t n_rays,
                                       const int32_t *ids, int32_t n_ids, const float *mlp, float ert_eps,
                                       const float *aux, const float *dL_drgb, float *const *grad_grid,
                                       float *const *grad_planes, float *grad_mlp, void *stream);

/* Gradients of the ray-batch render with per-block MLPs (cow_render_rays
 * with COW_FLAG_BLOCK_MLPS, no early termination): the adjoint of Eq. 5 with
 * Eq. 3 per block (Sec. 4.1 Phi^{k,l}) and Eq. 11 inside each block, with
 * respect to every grid and plane feature and every parameter of the MLPs
 * of the blocks in ids, given dL/dC per ray.  Each ray is marched twice
 * (once for every block's C^k, F^k and transmittance, once to scatter);
 * between the two, one thread per (ray, block) back-propagates that block's
 * MLP.  Occupancy is held fixed.
 *   o, d, ids, n_ids : as the forward call (device o, d);
 *   dL_drgb          : device float32 n_rays x 3;
 *   grad_grid, grad_planes : as cow_render_backward (accumulated);
 *   grad_block_mlps  : device float32 n_blocks x block_mlp_nparam(n_freq)
 *                      (the layout cow_set_block_mlps takes), accumulated;
 *                      rows of blocks not in ids are not touched.
 * Scratch: 64 bytes per (ray, block of ids) of device memory, kept by the
 * context.  Floating-point sums over rays are in no fixed order.
 * Errors: INVALID_ARG (no per-block MLPs set, bad ids, host or misaligned
 * arrays), OOM, CUDA; resident blocks as cow_render. */
cow_status cow_render_backward_block_mlps(cow_ctx *ctx, const float *o, const float *d, int64_t n_rays,
                                          const int32_t *ids, int32_t n_ids, const float *dL_drgb,
                                          float *const *grad_grid, float *const *grad_planes, float *grad_block_mlps,
                                          void *stream);

/* The same gradients without the backward's first march.  The forward
 * cow_render_rays_block_state renders like cow_render_rays with
 * COW_FLAG_BLOCK_MLPS and no early termination (Eq. 5 over the blocks' own
 * MLPs) and also writes, per (ray, block at its position in ids), what the
 * first march of the backward would compute: the block's C^k (3) and F^k (4)
 * and the transmittance in front of it (-1 when the block has no occupied
 * sample on the ray) -- out_state: device float32 n_rays x n_ids x 8,
 * 16-byte aligned.  cow_render_backward_block_mlps_state takes that state
 * (the same rays, ids and per-block MLPs, features unchanged since) and
 * marches once.  Scratch: 32 bytes per (ray, block of ids), kept by the
 * context.  Errors: as cow_render_rays / cow_render_backward_block_mlps;
 * INVALID_ARG for a null, host or misaligned state. */
cow_status cow_render_rays_block_state(cow_ctx *ctx, const float *o, const float *d, int64_t n_rays,
                                       const int32_t *ids, int32_t n_ids, float *out_rgb, float *out_state,
                                       void *stream);
cow_status cow_render_backward_block_mlps_state(cow_ctx *ctx, const float *o, const float *d, int64_t n_rays,
                                                const int32_t *ids, int32_t n_ids, const float *state,
                                                const float *dL_drgb, float *const *grad_grid,
                                                float *const *grad_planes, float *grad_block_mlps, void *stream);

/* Re-pack block `block`'s features from new FP32 masters (same layouts as
 * cow_block_desc; host or device, 16-byte aligned) into the context's
 * storage format; occupancy and z_top stay as loaded (the differentiation
 * form holds them fixed while the features are optimised). */
cow_status cow_update_features(cow_ctx *ctx, int32_t block, const float *grid, const float *plane_xy,
                               const float *plane_xz, const float *plane_yz, void *stream);

/* Training-stage regularisers of Sec. 4.3 on the loaded blocks, with their
 * gradients with respect to the density channel of the grids and planes.
 *   cow_sparsity_loss (Eq. 7): the mean over n_points points (device, FP32
 *     x, y, z) of alpha(p) = 1 - exp(-sigma(p) delta), sigma from the first
 *     block of ids that contains p (Eq. 4 membership), delta that block's
 *     sample spacing; a point in no block counts 0.  The paper draws the
 *     points uniformly in the scene's box (2^14 of them).
 *   cow_opacity_loss (Eq. 8): for each ray (device o, d as cow_render_rays,
 *     blocks ordered per ray) and each block with at least one occupied
 *     sample, the binary entropy -(a log a + (1 - a) log(1 - a)) of the
 *     block's opacity a = 1 - prod (1 - alpha_i) (Eq. 11), clamped to
 *     [1e-6, 1 - 1e-6]; the mean over rays of the sum over blocks.  No early
 *     termination.  block_T: NULL (every block is marched once for its
 *     opacity and once to scatter), or the out_block_T of a
 *     cow_render_rays_block_t call on the same rays and ids (one march).
 * Both add weight * loss to *loss (a device float; NULL: not computed) and
 * weight * d loss / d f0 into the FP32 gradient arrays, laid out as for
 * cow_render_backward (grad_grid / grad_planes both NULL: no gradient;
 * individual entries may be NULL).  ids: 1 .. 64 block ids.
 * Errors: INVALID_ARG, OOM (residency budget), CUDA. */
cow_status cow_sparsity_loss(cow_ctx *ctx, const float *points, int64_t n_points, const int32_t *ids, int32_t n_ids,
                             float weight, float *loss, float *const *grad_grid, float *const *grad_planes,
                             void *stream);
cow_status cow_opacity_loss(cow_ctx *ctx, const float *o, const float *d, int64_t n_rays, const int32_t *ids,
                            int32_t n_ids, const float *block_T, float weight, float *loss, float *const *grad_grid,
                            float *const *grad_planes, void *stream);

/* One Adam step on n FP32 parameters (device arrays param, grad, m, v):
 *   m = b1 m + (1-b1) g;  v = b2 v + (1-b2) g^2;
 *   param -= lr (m / (1 - b1^step)) / (sqrt(v / (1 - b2^step)) + eps). */
cow_status cow_adam_step(float *param, const float *grad, float *m, float *v, int64_t n, float lr, float beta1,
                         float beta2, float eps, int32_t step, void *stream);

/* Mean squared error of n values (device): dL_drgb = 2 (rgb - target) / n and,
 * when loss is not NULL, *loss (device float) = mean (rgb - target)^2. */
cow_status cow_mse_grad(const float *rgb, const float *target, int64_t n, float *dL_drgb, float *loss, void *stream);

/* Marching schedule of cow_render; all give the same image up to FP32
 * rounding (the oracle parity holds for each).
 *   COW_SCHED_THREAD: one ray per thread, a warp on an 8x4 pixel patch, so
 *     neighbouring rays share cache lines; each CTA copies its view's block
 *     records to shared memory with one TMA bulk copy;
 *   COW_SCHED_THREAD_CONST (default): the same marcher with the call's block
 *     records passed in the kernel's parameter buffer and read through the
 *     constant cache, which leaves the L1 data pipe to the feature gathers
 *     (measured 4 % faster at 1080p); used when the call's views select at
 *     most 96 block records in total, otherwise the call runs as
 *     COW_SCHED_THREAD;
 *   COW_SCHED_WARP: one ray per warp, the 32 lanes on 32 consecutive lattice
 *     samples of that ray, the in-block weights of Eq. 1 as a prefix product
 *     across the lanes (measured slower on aerial views: rays of one tile are
 *     marched one after another, so their texels are fetched again).
 * Errors: INVALID_ARG for a null context or an unknown schedule. */
#define COW_SCHED_WARP 0
#define COW_SCHED_THREAD 1
#define COW_SCHED_THREAD_CONST 2
cow_status cow_set_schedule(cow_ctx *ctx, int32_t schedule);

/* Processing order of the ray-batch calls (cow_render_rays,
 * cow_render_rays_block_t, cow_render_partials, cow_render_backward,
 * cow_render_backward_block_mlps, cow_opacity_loss).  COW_RAY_ORDER_COHERENT (default): a
 * batch of at least 8192 rays is marched in a coherent order -- rays grouped
 * by the cell of their entry into the call's blocks' bounding box (8 x 8 x 8)
 * and of their direction (8 x 8 x 8), by a counting sort on the device -- so
 * that the rays of one warp gather neighbouring texels; random training rays
 * otherwise send every lane of a warp to a different line (measured on 2^20
 * random rays over 2x2 blocks of 128^3 / 512^2 FP32 features: forward 75.8
 * -> 44.3 ms, backward 170 -> 135 ms).  COW_RAY_ORDER_GIVEN: thread t marches
 * ray t.  Outputs are written at each ray's own index either way and each
 * ray's values are the same; gradient sums change only by the order of their
 * FP32 reductions.  The order costs a key pass, a scan and a scatter (about
 * 12 bytes a ray and 1 MiB of context scratch).  Errors: INVALID_ARG. */
#define COW_RAY_ORDER_GIVEN 0
#define COW_RAY_ORDER_COHERENT 1
cow_status cow_set_ray_order(cow_ctx *ctx, int32_t mode);

/* Order in which cow_render launches the screen tiles of a view (the image is
 * the same): 0 = raster order; k > 0 = vertical strips of k tile columns,
 * each walked row by row, so the tiles in flight cover a compact screen
 * region (their rays share more texels in L2).  Errors: INVALID_ARG. */
cow_status cow_set_tile_order(cow_ctx *ctx, int32_t strip_tiles);

/* Autotuner of cow_render's marching schedule: renders the given views
 * (arguments as cow_render, device outputs only: out_rgb is overwritten)
 * with every schedule (COW_SCHED_THREAD_CONST, COW_SCHED_THREAD,
 * COW_SCHED_WARP) and tile order (raster, strips of 2 and 4 tile columns),
 * reps timed renders each after one warm-up, keeps the fastest on the
 * context and reports it (any out pointer may be NULL).
 * Errors: as cow_render. */
cow_status cow_tune_schedule(cow_ctx *ctx, const cow_camera *cams, int32_t n_views, const int32_t *ids,
                             const int32_t *ids_offsets, const float *mlp, float ert_eps, uint32_t flags,
                             float *out_rgb, int32_t reps, void *stream, int32_t *out_schedule,
                             int32_t *out_strip, float *out_ms);

/* Wait for the stream and report a device-side error word set by a kernel of
 * this context (COW_ERR_DEVICE_ASSERT or COW_ERR_TIMEOUT); clears it. */
cow_status cow_sync_check(cow_ctx *ctx, void *stream);

/* Test hook (no counterpart in the paper): lets a test drive the bounded
 * device-side waits to their time-out without faulting anything.  The
 * kernels that stage a view's block records into shared memory with a TMA
 * bulk copy (the COW_SCHED_THREAD and COW_SCHED_WARP view schedules and the
 * batched form) wait for it on an mbarrier with an iteration limit.  With
 * COW_TEST_SKIP_RECORD_COPY the copy is not issued, so the barrier's phase
 * never completes and nothing is in flight; each wait gives up after
 * wait_polls polls (0 = the default 2^24), the kernel records the time-out
 * (cow_sync_check then returns COW_ERR_TIMEOUT), its CTAs leave without
 * writing their pixels, and the context stays usable.  Production callers
 * never call this (flags 0, wait_polls 0).  Errors: INVALID_ARG. */
#define COW_TEST_SKIP_RECORD_COPY 1u
cow_status cow_set_test_hooks(cow_ctx *ctx, uint32_t flags, uint32_t wait_polls);

/* Copy out a block's occupancy bits (ceil(ncell/32) words, cell index
 * (cz*Nc + cy)*Nc + cx, bit c&31 of word c>>5) into host memory. */
cow_status cow_export_occupancy(const cow_ctx *ctx, int32_t block, uint32_t *out_bits, int64_t n_words);

/* Copy out the coarse level of a block's two-level occupancy grid (Sec. 4.1,
 * the multi-level occupancy grid psi^{k,l}): coarse cell (gx, gy, gz) covers
 * occupancy cells [4g, 4g + 3] per axis (clipped at Nc) and its bit is the OR
 * of theirs.  Nc2 = ceil(Nc / 4) per axis, index (gz*Nc2 + gy)*Nc2 + gx, bit
 * g&31 of word g>>5; ceil(Nc2^3 / 32) words into host memory.  The marcher
 * tests this bit first and leaves an empty coarse cell in one exact jump.
 * Errors: INVALID_ARG (bad block, n_words too small), CUDA. */
cow_status cow_export_occupancy_coarse(const cow_ctx *ctx, int32_t block, uint32_t *out_bits, int64_t n_words);

/* Copy out a block's packed tensor (0 = grid, 1..3 = planes xy, xz, yz) in its
 * storage format into host memory, with its 8 per-channel scale exponents.
 * The output is in the natural layout (vertex after vertex, nbytes >=
 * count x 8 x element size).  On the device FP16 / BF16 / FP8 are held in a
 * pair layout (each element also carries the next vertex of its row, so one
 * 32- or 16-byte load returns both corners of an interpolation pair): twice
 * the memory of the natural layout.  For COW_FP8_BF16D, tensor 0 is the FP8
 * grid (all 8 channels; the kernels read channel 0 from tensor 4) and tensor
 * 4 the grid's BF16 channel 0, one value per vertex (scale exponents 0).
 * Errors: INVALID_ARG (block or tensor out of range, nbytes too small),
 * UNSUPPORTED (the grid of a brick-sparse context), CUDA. */
cow_status cow_export_packed(const cow_ctx *ctx, int32_t block, int32_t tensor, void *out, int64_t nbytes,
                             int32_t *out_scale_exp);

/* Measurement aid (no counterpart in the paper): the throughput of random
 * aligned gathers of bytes_per_load (16 or 32) bytes by every thread of a
 * full-GPU launch from a device buffer of buffer_bytes (a power of two, 1 KiB
 * to 64 GiB), in useful GB/s -- the access pattern of the marcher's texel
 * gathers.  A buffer that fits L1 gives the L1 scattered-gather rate, tens of
 * MB the L2 rate, GBs the HBM rate: the denominators of the marcher's gather
 * roofline.  Allocates and frees its buffer; synchronises `stream`.
 * Errors: INVALID_ARG, OOM, CUDA. */
cow_status cow_gather_peak(int32_t bytes_per_load, int64_t buffer_bytes, int32_t iters, double *out_gbs,
                           void *stream);

/* Measurement aid (no counterpart in the paper): the rate of random,
 * 16-byte-aligned non-returning 4-float reductions (red.global.add.v4.f32,
 * the backward's scatter) by every thread of a full-GPU launch into a device
 * buffer of buffer_bytes (a power of two, 1 KiB to 64 GiB), in 10^9
 * reductions per second.  A buffer that fits L2 gives the L2 reduction rate.
 * Allocates and frees its buffer; synchronises `stream`.  Errors:
 * INVALID_ARG, OOM, CUDA. */
cow_status cow_reduce_peak(int64_t buffer_bytes, int32_t iters, double *out_gred_per_s, void *stream);

/* Message of the last failed call on this thread ("" if none). */
const char *cow_last_error(void);

/* ABI version of this library. */
int32_t cow_version(void);

#ifdef __cplusplus
}
#endif
#endif /* COW_H */
