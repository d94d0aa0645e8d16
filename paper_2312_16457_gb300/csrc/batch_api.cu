// batch_api.cu -- C ABI of the batched form: many cameras of uneven size and
// LOD set served by one persistent launch (K8), optionally replayed from a
// CUDA graph, with the tile shape and the number of resident CTAs picked by
// an autotuner that times the candidates on the batch itself.  Under a
// residency budget the views are served in groups whose blocks fit the
// budget together: one launch per group, its blocks made resident first.
#include <algorithm>
#include <cstring>
#include <vector>

#include "cow_internal.h"

using namespace cowi;

struct cow_batch {
    cow_ctx *ctx = nullptr;
    int device = 0;
    int32_t max_views = 0, max_ids = 0;
    // staging: [hdr 256 B | views max_views x ViewRec | recs max_ids x BlockRec]
    size_t stage_bytes = 0, views_off = 256, recs_off = 0;
    unsigned char *h_stage = nullptr;  // pinned
    unsigned char *d_stage = nullptr;
    unsigned *d_counter = nullptr;
    cudaEvent_t copied = nullptr;      // the last H2D copy of h_stage has run
    cudaStream_t cap_stream = nullptr; // stream for graph capture
    // views of the current batch
    std::vector<cow_camera> cams;
    std::vector<int32_t> ids, offs;
    int64_t n_pixels = 0;
    int32_t n_items = 0;
    int32_t max_blk = 0;               // longest block list of a view
    bool dirty = true;                 // staging must be rebuilt
    uint64_t rec_gen = 0;              // the context's record generation the staging holds
    int32_t last_groups = 0;           // launches of the last render (groups under a budget)
    bool backward = false;             // under a budget: the next render serves the views last to first
    int tile_cfg = 0, ctas_per_sm = 4; // launch configuration (autotuned)
    float run_frac = 0.5f;             // under a budget: a run's blocks fill at most this fraction of it
    int records = COW_BATCH_RECORDS_PARAM;  // record placement (cow_batch_set_records)
    int sched = COW_BATCH_SCHED_QUEUE;      // persistent queue, or the view marcher's grid (cow_batch_set_schedule)
    int sms = 0;
    // captured graph and the arguments it was captured with
    cudaGraphExec_t exec = nullptr;
    cow::BatchArgs gargs;
    int g_tile = -1, g_grid = -1;
    uint64_t g_gen = 0;
    // runs of views whose distinct blocks fit the launch parameter buffer:
    // one persistent launch a run, records by value (used when every view
    // has at most kParamRecs blocks and no residency budget is set)
    struct Run {
        size_t off = 0;           // the run's [hdr | views | index lists] in stage2
        int32_t n_views = 0, n_items = 0;
        cow::ParamRecs pr;        // its distinct blocks' records
    };
    std::vector<Run> runs;
    bool param_mode = false;
    size_t stage2_cap = 0, stage2_bytes = 0;
    unsigned char *h_stage2 = nullptr;  // pinned
    unsigned char *d_stage2 = nullptr;
    unsigned *d_counters = nullptr;     // one work-queue head per run
    int32_t counters_cap = 0;
    uint64_t stage_gen = 0;             // advances whenever a staging is rebuilt
};

namespace {

constexpr int kWarpItems = 4;  // tile_cfg of the warp-item kernel (8x4 pixels per warp)

void batch_destroy(cow_batch *b) {
    if (!b) return;
    DeviceGuard dg(b->device);
    if (b->exec) cudaGraphExecDestroy(b->exec);
    if (b->copied) cudaEventDestroy(b->copied);
    if (b->cap_stream) cudaStreamDestroy(b->cap_stream);
    cudaFreeHost(b->h_stage);
    cudaFree(b->d_stage);
    cudaFree(b->d_counter);
    cudaFreeHost(b->h_stage2);
    cudaFree(b->d_stage2);
    cudaFree(b->d_counters);
    delete b;
}

// Build the pinned staging (header, view records, block records) for the
// views first .. last-1 of the current cameras and the tile shape.  A view's
// pixels keep their place in the whole batch's output.
cow_status build_stage(cow_batch *b, int32_t first, int32_t last) {
    cudaError_t e = cudaEventSynchronize(b->copied);  // the previous copy has read h_stage
    if (e != cudaSuccess) return fail(COW_ERR_CUDA, "cudaEventSynchronize: %s", cudaGetErrorString(e));
    int tw, th;
    cow::batch_tile_shape(b->tile_cfg, &tw, &th);
    const int32_t nv = (int32_t)b->cams.size();
    cow::ViewRec *vr = (cow::ViewRec *)(b->h_stage + b->views_off);
    cow::BlockRec *br = (cow::BlockRec *)(b->h_stage + b->recs_off);
    int64_t tiles = 0, pix = 0;
    b->max_blk = 0;
    for (int32_t v = 0; v < first; v++) pix += (int64_t)b->cams[(size_t)v].width * b->cams[(size_t)v].height;
    const int32_t id0 = b->offs[(size_t)first];
    for (int32_t v = first; v < last; v++) {
        b->max_blk = std::max(b->max_blk, b->offs[(size_t)v + 1] - b->offs[(size_t)v]);
        const cow_camera &cam = b->cams[(size_t)v];
        cow::ViewRec &r = vr[v - first];
        std::memset(&r, 0, sizeof(r));
        for (int rr = 0; rr < 3; rr++) {
            for (int k = 0; k < 3; k++) r.Rm[3 * rr + k] = (float)cam.c2w[4 * rr + k];
            r.o[rr] = (float)cam.c2w[4 * rr + 3];
        }
        r.f = (float)focal_length(cam.height, cam.fov_y_deg);
        r.W = cam.width;
        r.H = cam.height;
        r.tiles_x = (cam.width + tw - 1) / tw;
        r.tile_begin = (int32_t)tiles;
        r.ids_begin = b->offs[(size_t)v] - id0;
        r.ids_count = b->offs[(size_t)v + 1] - b->offs[(size_t)v];
        r.pix_offset = pix;
        tiles += (int64_t)r.tiles_x * ((cam.height + th - 1) / th);
        pix += (int64_t)cam.width * cam.height;
    }
    if (tiles > 0x7fffffff) return fail(COW_ERR_INVALID_ARG, "too many tiles in one batch");
    for (int32_t k = id0; k < b->offs[(size_t)last]; k++) br[k - id0] = b->ctx->recs[(size_t)b->ids[(size_t)k]];
    int32_t *hdr = (int32_t *)b->h_stage;
    hdr[0] = last - first;
    hdr[1] = (int32_t)tiles;
    b->n_items = (int32_t)tiles;
    b->n_pixels = 0;
    for (int32_t v = 0; v < nv; v++) b->n_pixels += (int64_t)b->cams[(size_t)v].width * b->cams[(size_t)v].height;
    b->rec_gen = b->ctx->rec_gen;
    b->dirty = first != 0 || last != nv;  // a group's staging: the whole batch must be rebuilt later
    b->param_mode = false;
    b->stage_gen++;
    return COW_OK;
}

// Views in runs whose distinct blocks fit a launch's parameter buffer
// (kParamRecs records): a run grows by the view that adds the fewest new
// blocks (in view order for very large batches) while the union still fits.
// Every run gets its records by value and its views' lists as byte indices
// into them; the staging of all runs is one pinned buffer copied at once.
cow_status build_runs(cow_batch *b, int32_t first, int32_t last) {
    cudaError_t e = cudaEventSynchronize(b->copied);  // the previous copy has read the stagings
    if (e != cudaSuccess) return fail(COW_ERR_CUDA, "cudaEventSynchronize: %s", cudaGetErrorString(e));
    int tw, th;
    cow::batch_tile_shape(b->tile_cfg, &tw, &th);
    const int32_t nv = (int32_t)b->cams.size();
    const int32_t nb = (int32_t)b->ctx->blocks.size();
    // distinct blocks of every view
    std::vector<std::vector<int32_t>> own((size_t)nv);
    for (int32_t v = 0; v < nv; v++) {
        for (int32_t k = b->offs[(size_t)v]; k < b->offs[(size_t)v + 1]; k++) {
            const int32_t id = b->ids[(size_t)k];
            if (std::find(own[(size_t)v].begin(), own[(size_t)v].end(), id) == own[(size_t)v].end())
                own[(size_t)v].push_back(id);
        }
    }
    std::vector<std::vector<int32_t>> run_views;
    {
        // views outside [first, last) count as done
        std::vector<char> done((size_t)nv, 1), in((size_t)nb, 0);
        for (int32_t v = first; v < last; v++) done[(size_t)v] = 0;
        const bool pick_best = last - first <= 1024;
        int32_t left = last - first, next = first;
        while (left > 0) {
            std::vector<int32_t> views, blocks;
            for (;;) {
                int32_t best = -1, best_add = 1 << 30;
                if (views.empty() || !pick_best) {
                    while (next < nv && done[(size_t)next]) next++;
                    if (next < nv) {
                        int32_t add = 0;
                        for (int32_t id : own[(size_t)next]) add += in[(size_t)id] ? 0 : 1;
                        best = next;
                        best_add = add;
                    }
                } else {
                    for (int32_t v = 0; v < nv; v++) {
                        if (done[(size_t)v]) continue;
                        int32_t add = 0;
                        for (int32_t id : own[(size_t)v]) add += in[(size_t)id] ? 0 : 1;
                        if (add < best_add) {
                            best_add = add;
                            best = v;
                        }
                    }
                }
                if (best < 0 || (int32_t)blocks.size() + best_add > cow::kParamRecs) break;
                done[(size_t)best] = 1;
                left--;
                views.push_back(best);
                for (int32_t id : own[(size_t)best])
                    if (!in[(size_t)id]) {
                        in[(size_t)id] = 1;
                        blocks.push_back(id);
                    }
            }
            for (int32_t id : blocks) in[(size_t)id] = 0;
            run_views.push_back(std::move(views));
        }
    }
    // staging: per run [hdr 256 B | views | index bytes], 256-byte aligned
    size_t need = 0;
    for (const auto &rv : run_views) {
        size_t ni = 0;
        for (int32_t v : rv) ni += (size_t)(b->offs[(size_t)v + 1] - b->offs[(size_t)v]);
        need += 256 + ((rv.size() * sizeof(cow::ViewRec) + 255) & ~(size_t)255) + ((ni + 255) & ~(size_t)255);
    }
    if (need > b->stage2_cap) {
        cudaFreeHost(b->h_stage2);
        cudaFree(b->d_stage2);
        b->h_stage2 = nullptr;
        b->d_stage2 = nullptr;
        b->stage2_cap = 0;
        e = cudaHostAlloc((void **)&b->h_stage2, need, cudaHostAllocDefault);
        if (e == cudaSuccess) e = cudaMalloc((void **)&b->d_stage2, need);
        if (e != cudaSuccess)
            return fail(e == cudaErrorMemoryAllocation ? COW_ERR_OOM : COW_ERR_CUDA, "batch staging: %s",
                        cudaGetErrorString(e));
        b->stage2_cap = need;
    }
    if ((int32_t)run_views.size() > b->counters_cap) {
        cudaFree(b->d_counters);
        b->d_counters = nullptr;
        b->counters_cap = 0;
        e = cudaMalloc((void **)&b->d_counters, run_views.size() * sizeof(unsigned));
        if (e != cudaSuccess)
            return fail(e == cudaErrorMemoryAllocation ? COW_ERR_OOM : COW_ERR_CUDA, "batch counters: %s",
                        cudaGetErrorString(e));
        b->counters_cap = (int32_t)run_views.size();
    }
    std::vector<int64_t> pix_of((size_t)nv + 1, 0);
    for (int32_t v = 0; v < nv; v++)
        pix_of[(size_t)v + 1] = pix_of[(size_t)v] + (int64_t)b->cams[(size_t)v].width * b->cams[(size_t)v].height;
    b->runs.assign(run_views.size(), cow_batch::Run());
    std::vector<int32_t> slot((size_t)nb, -1);
    size_t off = 0;
    int64_t total_items = 0;
    b->max_blk = 0;
    for (size_t r = 0; r < run_views.size(); r++) {
        cow_batch::Run &run = b->runs[r];
        const auto &rv = run_views[r];
        run.off = off;
        run.n_views = (int32_t)rv.size();
        std::memset(&run.pr, 0, sizeof(run.pr));
        int32_t n_rec = 0;
        std::vector<int32_t> used;
        cow::ViewRec *vr = (cow::ViewRec *)(b->h_stage2 + off + 256);
        unsigned char *idx = b->h_stage2 + off + 256 + ((rv.size() * sizeof(cow::ViewRec) + 255) & ~(size_t)255);
        int64_t tiles = 0;
        int32_t n_idx = 0;
        for (size_t k = 0; k < rv.size(); k++) {
            const int32_t v = rv[k];
            const cow_camera &cam = b->cams[(size_t)v];
            cow::ViewRec &w = vr[k];
            std::memset(&w, 0, sizeof(w));
            for (int rr = 0; rr < 3; rr++) {
                for (int q = 0; q < 3; q++) w.Rm[3 * rr + q] = (float)cam.c2w[4 * rr + q];
                w.o[rr] = (float)cam.c2w[4 * rr + 3];
            }
            w.f = (float)focal_length(cam.height, cam.fov_y_deg);
            w.W = cam.width;
            w.H = cam.height;
            w.tiles_x = (cam.width + tw - 1) / tw;
            w.tile_begin = (int32_t)tiles;
            w.ids_begin = n_idx;
            w.ids_count = b->offs[(size_t)v + 1] - b->offs[(size_t)v];
            w.pix_offset = pix_of[(size_t)v];
            b->max_blk = std::max(b->max_blk, w.ids_count);
            tiles += (int64_t)w.tiles_x * ((cam.height + th - 1) / th);
            for (int32_t q = b->offs[(size_t)v]; q < b->offs[(size_t)v + 1]; q++) {
                const int32_t id = b->ids[(size_t)q];
                if (slot[(size_t)id] < 0) {
                    slot[(size_t)id] = n_rec;
                    run.pr.r[n_rec++] = b->ctx->recs[(size_t)id];
                    used.push_back(id);
                }
                idx[n_idx++] = (unsigned char)slot[(size_t)id];
            }
        }
        for (int32_t id : used) slot[(size_t)id] = -1;
        if (tiles > 0x7fffffff) return fail(COW_ERR_INVALID_ARG, "too many tiles in one batch run");
        int32_t *hdr = (int32_t *)(b->h_stage2 + off);
        hdr[0] = run.n_views;
        hdr[1] = (int32_t)tiles;
        run.n_items = (int32_t)tiles;
        total_items += tiles;
        off += 256 + ((rv.size() * sizeof(cow::ViewRec) + 255) & ~(size_t)255) + (((size_t)n_idx + 255) & ~(size_t)255);
    }
    b->stage2_bytes = off;
    b->n_pixels = pix_of[(size_t)nv];
    b->n_items = (int32_t)std::min<int64_t>(total_items, 0x7fffffff);
    b->rec_gen = b->ctx->rec_gen;
    b->dirty = first != 0 || last != nv;  // a budget run's staging: the whole batch must be rebuilt later
    b->param_mode = true;
    b->stage_gen++;
    return COW_OK;
}

// Every view's list (of views first .. last-1, or all) fits a launch's
// parameter buffer.
bool runs_fit(const cow_batch *b, int32_t first = 0, int32_t last = -1) {
    if (last < 0) last = (int32_t)b->offs.size() - 1;
    for (int32_t v = first; v < last; v++)
        if (b->offs[(size_t)v + 1] - b->offs[(size_t)v] > cow::kParamRecs) return false;
    return true;
}

cow::BatchArgs make_args(cow_batch *b, const float *mlp, float ert_eps, uint32_t flags, float *rgb, float *aux,
                         int32_t *ns) {
    cow::BatchArgs a;
    std::memset(&a, 0, sizeof(a));
    a.hdr = (const int32_t *)b->d_stage;
    a.views = (const cow::ViewRec *)(b->d_stage + b->views_off);
    a.recs = (const cow::BlockRec *)(b->d_stage + b->recs_off);
    a.mlp = mlp;
    a.ert_eps = ert_eps;
    a.flags = flags;
    a.dtype = kernel_dtype(b->ctx);
    a.smem_recs = b->max_blk <= 96 ? b->max_blk : 0;  // longer lists are read from global memory
    a.out_rgb = rgb;
    a.out_aux = aux;
    a.out_nsamp = ns;
    a.err = b->ctx->d_err;
    a.counter = b->d_counter;
    a.test_flags = b->ctx->test_flags;
    a.wait_polls = b->ctx->wait_polls;
    return a;
}

// The batch on one stream: staging copy, queue reset, persistent launch.
// `mark` records b->copied after the copy (not inside a graph capture: a
// captured event cannot be waited on from outside; graph launches record it
// after the whole graph instead).
cudaError_t enqueue(cow_batch *b, const cow::BatchArgs &a, int tile_cfg, int grid, cudaStream_t st, bool mark) {
    if (b->param_mode) {  // all runs: one staging copy, the queue heads, one launch a run
        cudaError_t e = cudaMemcpyAsync(b->d_stage2, b->h_stage2, b->stage2_bytes, cudaMemcpyHostToDevice, st);
        if (e == cudaSuccess && mark) e = cudaEventRecord(b->copied, st);
        if (e == cudaSuccess) e = cudaMemsetAsync(b->d_counters, 0, b->runs.size() * sizeof(unsigned), st);
        for (size_t r = 0; r < b->runs.size() && e == cudaSuccess; r++) {
            const cow_batch::Run &run = b->runs[r];
            if (run.n_items == 0) continue;
            cow::BatchArgs ar = a;
            ar.hdr = (const int32_t *)(b->d_stage2 + run.off);
            ar.views = (const cow::ViewRec *)(b->d_stage2 + run.off + 256);
            ar.vidx = b->d_stage2 + run.off + 256 + (((size_t)run.n_views * sizeof(cow::ViewRec) + 255) & ~(size_t)255);
            ar.recs = nullptr;
            ar.smem_recs = 0;
            ar.counter = b->d_counters + r;
            e = cow::launch_march_batch(ar, tile_cfg, grid, st, &run.pr);
        }
        return e;
    }
    cudaError_t e = cudaMemcpyAsync(b->d_stage, b->h_stage, b->stage_bytes, cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess && mark) e = cudaEventRecord(b->copied, st);
    if (e == cudaSuccess) e = cudaMemsetAsync(b->d_counter, 0, sizeof(unsigned), st);
    if (e == cudaSuccess) e = cow::launch_march_batch(a, tile_cfg, grid, st);
    return e;
}

// Under a residency budget: cut the views, in the batch's order, into runs
// whose blocks fit a fraction of the budget together (a view joins the
// current run while the run's distinct blocks plus its own still fit; a view
// alone above that fraction forms its own run), make each run's blocks
// resident (LRU unloading of the others) and launch the persistent kernel on
// that run.  With runs of at most half the budget a run's loads unload only
// blocks of earlier runs, so they proceed on the copy stream while the
// previous run marches.  Successive renders walk the views in alternating
// directions, so a render starts with the blocks the previous one left
// resident.  Runs are launched eagerly on the caller's stream, never from the
// graph: each one rewrites the staging and the block records.
cow_status render_groups(cow_batch *b, const float *mlp, float ert_eps, uint32_t flags, float *rgb, float *aux,
                         int32_t *ns, cudaStream_t st) {
    cow_ctx *c = b->ctx;
    const int32_t nv = (int32_t)b->cams.size();
    const int32_t nb = (int32_t)c->blocks.size();
    const bool back = b->backward;
    std::vector<char> in((size_t)nb, 0);
    std::vector<int32_t> run_ids;
    int64_t run_bytes = 0;
    int32_t first = 0, groups = 0;  // first: the run's first view in walking order (step index)
    auto view_at = [&](int32_t k) { return back ? nv - 1 - k : k; };
    auto launch = [&](int32_t last) -> cow_status {  // steps first .. last-1
        cow_status rc = make_resident(c, run_ids.data(), (int64_t)run_ids.size(), st);
        if (rc != COW_OK) return rc;
        const int32_t lo = back ? nv - last : first, hi = back ? nv - first : last;
        // the run's views in sub-runs with records in the parameter buffer
        // when their lists fit, else one launch staging records in shared memory
        const bool param = b->records == COW_BATCH_RECORDS_PARAM && runs_fit(b, lo, hi);
        if (b->tile_cfg == kWarpItems && !param)
            return fail(COW_ERR_UNSUPPORTED, "warp items (tile_cfg 4) need records in the parameter buffer");
        if ((rc = param ? build_runs(b, lo, hi) : build_stage(b, lo, hi)) != COW_OK) return rc;
        const cow::BatchArgs a = make_args(b, mlp, ert_eps, flags, rgb, aux, ns);
        COW_CUDA(enqueue(b, a, b->tile_cfg, std::max(1, b->sms * b->ctas_per_sm), st, true));
        if ((rc = note_use(c, run_ids.data(), (int64_t)run_ids.size(), st)) != COW_OK) return rc;
        groups++;
        return COW_OK;
    };
    for (int32_t k = 0; k < nv; k++) {
        const int32_t v = view_at(k);
        // the view's distinct blocks, and the bytes it adds to the current run
        std::vector<int32_t> own;
        int64_t own_bytes = 0, add = 0;
        for (int32_t q = b->offs[(size_t)v]; q < b->offs[(size_t)v + 1]; q++) {
            const int32_t id = b->ids[(size_t)q];
            if (std::find(own.begin(), own.end(), id) != own.end()) continue;
            own.push_back(id);
            const int64_t by = block_feature_bytes(c, id);
            own_bytes += by;
            if (!in[(size_t)id]) add += by;
        }
        if (own_bytes > c->budget)
            return fail(COW_ERR_OOM, "batch view %d needs %lld bytes, over the residency budget of %lld", v,
                        (long long)own_bytes, (long long)c->budget);
        const int64_t cap = std::max<int64_t>(1, (int64_t)((double)c->budget * (double)b->run_frac));
        if (k > first && run_bytes + add > cap) {
            cow_status rc = launch(k);
            if (rc != COW_OK) return rc;
            for (int32_t id : run_ids) in[(size_t)id] = 0;
            run_ids.clear();
            run_bytes = 0;
            first = k;
            add = own_bytes;
        }
        for (int32_t id : own)
            if (!in[(size_t)id]) {
                in[(size_t)id] = 1;
                run_ids.push_back(id);
            }
        run_bytes += add;
    }
    cow_status rc = launch(nv);
    if (rc != COW_OK) return rc;
    b->last_groups = groups;
    b->backward = !back;
    return COW_OK;
}

// The grid schedule: the views in groups whose block lists, concatenated,
// fit one launch's parameter buffer, each group one launch of the view
// marcher (cow_render: one CTA per 16x8 tile, scheduled by the hardware);
// a view with a longer list forms its own group.  Outputs keep each view's
// place in the batch.
cow_status render_grid(cow_batch *b, const float *mlp, float ert_eps, uint32_t flags, float *rgb, float *aux,
                       int32_t *ns, cudaStream_t st) {
    const int32_t nv = (int32_t)b->cams.size();
    int64_t pix = 0;
    int32_t groups = 0;
    std::vector<int32_t> offs;
    for (int32_t v0 = 0; v0 < nv;) {
        int32_t v1 = v0 + 1;
        while (v1 < nv && b->offs[(size_t)v1 + 1] - b->offs[(size_t)v0] <= cow::kParamRecs) v1++;
        offs.assign((size_t)(v1 - v0) + 1, 0);
        int64_t gpix = 0;
        for (int32_t v = v0; v < v1; v++) {
            offs[(size_t)(v - v0) + 1] = b->offs[(size_t)v + 1] - b->offs[(size_t)v0];
            gpix += (int64_t)b->cams[(size_t)v].width * b->cams[(size_t)v].height;
        }
        cow_status rc = cow_render(b->ctx, b->cams.data() + v0, v1 - v0, b->ids.data() + b->offs[(size_t)v0], offs.data(),
                                   mlp, ert_eps, flags, rgb + 3 * pix, aux ? aux + 8 * pix : nullptr,
                                   ns ? ns + pix : nullptr, st);
        if (rc != COW_OK) return rc;
        pix += gpix;
        groups++;
        v0 = v1;
    }
    b->last_groups = groups;
    return COW_OK;
}

}  // namespace

namespace cowi {

void batch_detach(cow_batch *b) {
    if (b) b->ctx = nullptr;
}

}  // namespace cowi

extern "C" {

cow_status cow_batch_create(cow_ctx *ctx, int32_t max_views, int32_t max_ids, cow_batch **out) {
    g_last_error.clear();
    if (!ctx || !out || max_views < 1 || max_ids < 0 || max_views > (1 << 16) || max_ids > (1 << 22))
        return fail(COW_ERR_INVALID_ARG, "cow_batch_create: bad argument");
    *out = nullptr;
    DeviceGuard dg(ctx->device);
    cow_batch *b = new cow_batch();
    b->ctx = ctx;
    b->device = ctx->device;
    b->max_views = max_views;
    b->max_ids = max_ids;
    b->recs_off = (b->views_off + (size_t)max_views * sizeof(cow::ViewRec) + 255) & ~(size_t)255;
    b->stage_bytes = b->recs_off + (size_t)std::max(max_ids, 1) * sizeof(cow::BlockRec);
    cudaError_t e = cudaHostAlloc((void **)&b->h_stage, b->stage_bytes, cudaHostAllocDefault);
    if (e == cudaSuccess) e = cudaMalloc((void **)&b->d_stage, b->stage_bytes);
    if (e == cudaSuccess) e = cudaMalloc((void **)&b->d_counter, sizeof(unsigned));
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&b->copied, cudaEventDisableTiming);
    if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&b->cap_stream, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&b->sms, cudaDevAttrMultiProcessorCount, ctx->device);
    if (e != cudaSuccess) {
        batch_destroy(b);
        return fail(e == cudaErrorMemoryAllocation ? COW_ERR_OOM : COW_ERR_CUDA, "cow_batch_create: %s",
                    cudaGetErrorString(e));
    }
    std::memset(b->h_stage, 0, b->stage_bytes);
    ctx->batches.push_back(b);
    *out = b;
    return COW_OK;
}

cow_status cow_batch_free(cow_batch *b) {
    if (b && b->ctx) {
        auto &v = b->ctx->batches;
        v.erase(std::remove(v.begin(), v.end(), b), v.end());
    }
    batch_destroy(b);
    return COW_OK;
}

cow_status cow_batch_set_views(cow_batch *b, const cow_camera *cams, int32_t n_views, const int32_t *ids,
                               const int32_t *ids_offsets, int64_t *out_pixels) {
    COW_NVTX("cow_batch_set_views");
    g_last_error.clear();
    if (b && !b->ctx) return fail(COW_ERR_INVALID_ARG, "the batch's context has been freed");
    if (!b || !cams || n_views < 1 || !ids_offsets) return fail(COW_ERR_INVALID_ARG, "cow_batch_set_views: null argument");
    if (n_views > b->max_views) return fail(COW_ERR_INVALID_ARG, "%d views exceed the batch's %d", n_views, b->max_views);
    const int32_t n_ids = ids_offsets[n_views];
    if (ids_offsets[0] != 0 || n_ids < 0 || n_ids > b->max_ids)
        return fail(COW_ERR_INVALID_ARG, "ids_offsets must start at 0 and end at most at %d", b->max_ids);
    if (n_ids > 0 && !ids) return fail(COW_ERR_INVALID_ARG, "null ids");
    const int32_t nb = (int32_t)b->ctx->blocks.size();
    for (int32_t v = 0; v < n_views; v++) {
        const cow_camera &c = cams[v];
        if (c.width < 1 || c.height < 1 || c.width > 32768 || c.height > 32768 || !(c.fov_y_deg > 0.0 && c.fov_y_deg < 180.0))
            return fail(COW_ERR_INVALID_ARG, "view %d: bad camera", v);
        if (ids_offsets[v + 1] < ids_offsets[v]) return fail(COW_ERR_INVALID_ARG, "ids_offsets must be non-decreasing");
    }
    for (int32_t k = 0; k < n_ids; k++)
        if (ids[k] < 0 || ids[k] >= nb) return fail(COW_ERR_INVALID_ARG, "block id %d out of range", ids[k]);
    DeviceGuard dg(b->ctx->device);
    b->cams.assign(cams, cams + n_views);
    b->ids.assign(ids, ids + n_ids);
    b->offs.assign(ids_offsets, ids_offsets + n_views + 1);
    b->backward = false;
    cow_status rc = build_stage(b, 0, n_views);
    if (rc != COW_OK) return rc;
    if (out_pixels) *out_pixels = b->n_pixels;
    return COW_OK;
}

cow_status cow_batch_render(cow_batch *b, const float *mlp, float ert_eps, uint32_t flags, float *out_rgb,
                            float *out_aux, int32_t *out_nsamp, int32_t use_graph, void *stream) {
    COW_NVTX("cow_batch_render");
    g_last_error.clear();
    if (b && !b->ctx) return fail(COW_ERR_INVALID_ARG, "the batch's context has been freed");
    if (!b || !mlp || !out_rgb) return fail(COW_ERR_INVALID_ARG, "cow_batch_render: null argument");
    if (b->cams.empty()) return fail(COW_ERR_INVALID_ARG, "cow_batch_render: no views set");
    if (!(ert_eps >= 0.0f && ert_eps < 1.0f)) return fail(COW_ERR_INVALID_ARG, "ert_eps must be in [0, 1)");
    if (flags & ~COW_FLAG_MLP_BF16) return fail(COW_ERR_INVALID_ARG, "unknown flags");
    for (const void *q : {(const void *)mlp, (const void *)out_rgb})
        if (!is_device_ptr(q)) return fail(COW_ERR_INVALID_ARG, "the MLP and the outputs must be device memory");
    if ((out_aux && (!is_device_ptr(out_aux) || ((uintptr_t)out_aux & 15u))) || (out_nsamp && !is_device_ptr(out_nsamp)))
        return fail(COW_ERR_INVALID_ARG, "aux / nsamp must be device memory (aux 16-byte aligned)");
    DeviceGuard dg(b->ctx->device);
    cudaStream_t st = (cudaStream_t)stream;
    if (b->ctx->budget > 0) return render_groups(b, mlp, ert_eps, flags, out_rgb, out_aux, out_nsamp, st);
    if (b->sched == COW_BATCH_SCHED_GRID) return render_grid(b, mlp, ert_eps, flags, out_rgb, out_aux, out_nsamp, st);
    const bool want_runs = b->records == COW_BATCH_RECORDS_PARAM && runs_fit(b);
    if (b->tile_cfg == kWarpItems && !want_runs)
        return fail(COW_ERR_UNSUPPORTED, "warp items (tile_cfg 4) need records in the parameter buffer "
                                         "(COW_BATCH_RECORDS_PARAM, every view at most 96 blocks)");
    if (b->dirty || b->rec_gen != b->ctx->rec_gen || b->param_mode != want_runs) {
        // new views, tile shape, or block records
        cow_status rc = want_runs ? build_runs(b, 0, (int32_t)b->cams.size()) : build_stage(b, 0, (int32_t)b->cams.size());
        if (rc != COW_OK) return rc;
    }
    b->last_groups = 1;
    const cow::BatchArgs a = make_args(b, mlp, ert_eps, flags, out_rgb, out_aux, out_nsamp);
    const int grid = std::max(1, b->sms * b->ctas_per_sm);
    if (!use_graph) {
        COW_CUDA(enqueue(b, a, b->tile_cfg, grid, st, true));
        return COW_OK;
    }
    const bool same = b->exec && b->g_tile == b->tile_cfg && b->g_grid == grid && b->g_gen == b->stage_gen &&
                      std::memcmp(&b->gargs, &a, sizeof(a)) == 0;
    if (!same) {
        if (b->exec) {
            cudaGraphExecDestroy(b->exec);
            b->exec = nullptr;
        }
        // capture on the batch's own stream: the caller's may be the legacy stream
        COW_CUDA(cudaStreamBeginCapture(b->cap_stream, cudaStreamCaptureModeThreadLocal));
        cudaError_t ce = enqueue(b, a, b->tile_cfg, grid, b->cap_stream, false);
        cudaGraph_t graph = nullptr;
        cudaError_t ee = cudaStreamEndCapture(b->cap_stream, &graph);
        if (ce != cudaSuccess || ee != cudaSuccess) {
            if (graph) cudaGraphDestroy(graph);
            return fail(COW_ERR_CUDA, "graph capture failed: %s", cudaGetErrorString(ce != cudaSuccess ? ce : ee));
        }
        cudaError_t ie = cudaGraphInstantiate(&b->exec, graph, 0);
        cudaGraphDestroy(graph);
        if (ie != cudaSuccess) return fail(COW_ERR_CUDA, "cudaGraphInstantiate: %s", cudaGetErrorString(ie));
        b->gargs = a;
        b->g_tile = b->tile_cfg;
        b->g_grid = grid;
        b->g_gen = b->stage_gen;
    }
    COW_CUDA(cudaGraphLaunch(b->exec, st));
    COW_CUDA(cudaEventRecord(b->copied, st));
    return COW_OK;
}

cow_status cow_batch_set_run_fraction(cow_batch *b, float frac) {
    g_last_error.clear();
    if (!b || !(frac > 0.0f && frac <= 1.0f)) return fail(COW_ERR_INVALID_ARG, "run fraction must be in (0, 1]");
    b->run_frac = frac;
    return COW_OK;
}

cow_status cow_batch_set_records(cow_batch *b, int32_t mode) {
    g_last_error.clear();
    if (!b || (mode != COW_BATCH_RECORDS_PARAM && mode != COW_BATCH_RECORDS_SHARED))
        return fail(COW_ERR_INVALID_ARG, "cow_batch_set_records: bad argument");
    b->records = mode;
    return COW_OK;
}

cow_status cow_batch_set_schedule(cow_batch *b, int32_t sched) {
    g_last_error.clear();
    if (!b || (sched != COW_BATCH_SCHED_QUEUE && sched != COW_BATCH_SCHED_GRID))
        return fail(COW_ERR_INVALID_ARG, "cow_batch_set_schedule: bad argument");
    b->sched = sched;
    return COW_OK;
}

cow_status cow_batch_get_schedule(const cow_batch *b, int32_t *out_sched) {
    if (!b || !out_sched) return fail(COW_ERR_INVALID_ARG, "cow_batch_get_schedule: null argument");
    *out_sched = b->sched;
    return COW_OK;
}

cow_status cow_batch_get_config(const cow_batch *b, int32_t *out_tile_cfg, int32_t *out_ctas_per_sm,
                                int32_t *out_records) {
    if (!b) return fail(COW_ERR_INVALID_ARG, "cow_batch_get_config: null batch");
    if (out_tile_cfg) *out_tile_cfg = b->tile_cfg;
    if (out_ctas_per_sm) *out_ctas_per_sm = b->ctas_per_sm;
    if (out_records) *out_records = b->records;
    return COW_OK;
}

cow_status cow_batch_last_groups(const cow_batch *b, int32_t *out_groups) {
    if (!b || !out_groups) return fail(COW_ERR_INVALID_ARG, "cow_batch_last_groups: null argument");
    *out_groups = b->last_groups;
    return COW_OK;
}

cow_status cow_batch_set_config(cow_batch *b, int32_t tile_cfg, int32_t ctas_per_sm) {
    if (!b || tile_cfg < 0 || tile_cfg > kWarpItems || ctas_per_sm < 1 || ctas_per_sm > 32)
        return fail(COW_ERR_INVALID_ARG, "cow_batch_set_config: bad argument");
    if (tile_cfg != b->tile_cfg) b->dirty = true;
    b->tile_cfg = tile_cfg;
    b->ctas_per_sm = ctas_per_sm;
    return COW_OK;
}

cow_status cow_batch_tune(cow_batch *b, const float *mlp, float ert_eps, uint32_t flags, float *out_rgb, int32_t reps,
                          void *stream, int32_t *out_tile_cfg, int32_t *out_ctas_per_sm, float *out_ms) {
    COW_NVTX("cow_batch_tune");
    g_last_error.clear();
    if (!b || !mlp || !out_rgb || reps < 1) return fail(COW_ERR_INVALID_ARG, "cow_batch_tune: bad argument");
    if (!b->ctx) return fail(COW_ERR_INVALID_ARG, "the batch's context has been freed");
    if (b->cams.empty()) return fail(COW_ERR_INVALID_ARG, "cow_batch_tune: no views set");
    DeviceGuard dg(b->ctx->device);
    cudaStream_t st = (cudaStream_t)stream;
    cudaEvent_t e0, e1;
    COW_CUDA(cudaEventCreate(&e0));
    COW_CUDA(cudaEventCreate(&e1));
    static const int kCtas[] = {2, 3, 4, 6, 8};
    const int sched0 = b->sched;
    b->sched = COW_BATCH_SCHED_QUEUE;  // the queue's configurations first
    float best = 3.0e38f;
    int best_t = b->tile_cfg, best_c = b->ctas_per_sm;
    cow_status rc = COW_OK;
    const bool warp_items = b->records == COW_BATCH_RECORDS_PARAM && runs_fit(b);
    for (int t = 0; t <= (warp_items ? kWarpItems : kWarpItems - 1) && rc == COW_OK; t++) {
        for (int c : kCtas) {
            rc = cow_batch_set_config(b, t, c);
            if (rc != COW_OK) break;
            rc = cow_batch_render(b, mlp, ert_eps, flags, out_rgb, nullptr, nullptr, 0, stream);  // warm-up
            if (rc != COW_OK) break;
            cudaEventRecord(e0, st);
            for (int r = 0; r < reps && rc == COW_OK; r++)
                rc = cow_batch_render(b, mlp, ert_eps, flags, out_rgb, nullptr, nullptr, 0, stream);
            cudaEventRecord(e1, st);
            if (cudaEventSynchronize(e1) != cudaSuccess) {
                rc = fail(COW_ERR_CUDA, "cow_batch_tune: synchronisation failed");
                break;
            }
            float ms = 0.f;
            cudaEventElapsedTime(&ms, e0, e1);
            ms /= (float)reps;
            if (ms < best) {
                best = ms;
                best_t = t;
                best_c = c;
            }
        }
    }
    // the record placement at the best tile and CTAs
    const int rec0 = b->records;
    int best_r = rec0;
    if (rc == COW_OK && best_t != kWarpItems) {
        const int other = rec0 == COW_BATCH_RECORDS_PARAM ? COW_BATCH_RECORDS_SHARED : COW_BATCH_RECORDS_PARAM;
        rc = cow_batch_set_config(b, best_t, best_c);
        if (rc == COW_OK) rc = cow_batch_set_records(b, other);
        if (rc == COW_OK) rc = cow_batch_render(b, mlp, ert_eps, flags, out_rgb, nullptr, nullptr, 0, stream);
        if (rc == COW_OK) {
            cudaEventRecord(e0, st);
            for (int r = 0; r < reps && rc == COW_OK; r++)
                rc = cow_batch_render(b, mlp, ert_eps, flags, out_rgb, nullptr, nullptr, 0, stream);
            cudaEventRecord(e1, st);
            if (cudaEventSynchronize(e1) != cudaSuccess) rc = fail(COW_ERR_CUDA, "cow_batch_tune: synchronisation failed");
        }
        if (rc == COW_OK) {
            float ms = 0.f;
            cudaEventElapsedTime(&ms, e0, e1);
            ms /= (float)reps;
            if (ms < best) {
                best = ms;
                best_r = other;
            }
        }
        b->records = best_r;
    }
    // the grid schedule (the view marcher, one launch per group of views);
    // not under a budget, where runs are cut by residency
    int best_s = COW_BATCH_SCHED_QUEUE;
    if (rc == COW_OK && b->ctx->budget == 0) {
        b->sched = COW_BATCH_SCHED_GRID;
        rc = cow_batch_render(b, mlp, ert_eps, flags, out_rgb, nullptr, nullptr, 0, stream);
        if (rc == COW_OK) {
            cudaEventRecord(e0, st);
            for (int r = 0; r < reps && rc == COW_OK; r++)
                rc = cow_batch_render(b, mlp, ert_eps, flags, out_rgb, nullptr, nullptr, 0, stream);
            cudaEventRecord(e1, st);
            if (cudaEventSynchronize(e1) != cudaSuccess) rc = fail(COW_ERR_CUDA, "cow_batch_tune: synchronisation failed");
        }
        if (rc == COW_OK) {
            float ms = 0.f;
            cudaEventElapsedTime(&ms, e0, e1);
            ms /= (float)reps;
            if (ms < best) {
                best = ms;
                best_s = COW_BATCH_SCHED_GRID;
            }
        }
    }
    b->sched = rc == COW_OK ? best_s : sched0;
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (rc != COW_OK) return rc;
    cow_batch_set_config(b, best_t, best_c);
    if (out_tile_cfg) *out_tile_cfg = best_t;
    if (out_ctas_per_sm) *out_ctas_per_sm = best_c;
    if (out_ms) *out_ms = best;
    return COW_OK;
}

}  // extern "C"
