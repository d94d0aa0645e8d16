// cow_api.cu -- the C ABI of libcow (declared in include/cow.h).
//
// Host side of the renderer: argument checks, the context that owns the
// packed device scene, LOD selection / visibility / depth sort of App. D in
// FP64 on the host, and the launches of the marcher.
#include <algorithm>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <mutex>
#include <string>
#include <vector>

#include "cow_internal.h"

namespace cowi {

thread_local std::string g_last_error;

cow_status fail(cow_status st, const char *fmt, ...) {
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof(buf), fmt, ap);
    va_end(ap);
    g_last_error = buf;
    return st;
}

bool is_device_ptr(const void *p) {
    cudaPointerAttributes at;
    if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return at.type == cudaMemoryTypeDevice || at.type == cudaMemoryTypeManaged;
}

}  // namespace cowi

using namespace cowi;

namespace {

// storage of tensor t (0 grid, 1-3 planes) of a context: the mixed format
// keeps the grid in BF16 and the planes in FP8; the FP8 format with BF16
// density stores every tensor in FP8 (the grid's channel 0 again in BF16)
int tensor_dtype(int dtype, int t) {
    if (dtype == COW_BF16_FP8) return t == 0 ? COW_BF16 : COW_FP8_E4M3;
    if (dtype == COW_FP8_BF16D) return COW_FP8_E4M3;
    return dtype;
}

int elem_bytes(int dtype) { return dtype == COW_FP32 ? 4 : dtype == COW_FP8_E4M3 ? 1 : 2; }

// bytes of one packed element: an FP32 vertex, a pair of 16- or 8-bit
// vertices, or a 2x2 quad of FP8 vertices / texels (the planes of the mixed
// format, the grid and planes of the FP8 format with BF16 density) -- 32
// bytes for every format but pure FP8 (16)
int64_t packed_elem_bytes(int dtype) {
    return dtype == COW_FP32 || dtype == COW_BF16_FP8 || dtype == COW_FP8_BF16D ? 32 : 2 * 8 * elem_bytes(dtype);
}

// element layout of the grid (k_pack_grid) and its element counts per brick
// axis (the layout's halo: a paired axis needs no extra element)
int grid_layout(int dtype) {
    return dtype == COW_FP32 ? cow::kLayNat : dtype == COW_FP8_BF16D ? cow::kLayQuad8 : cow::kLayPair;
}
void brick_dims(int dtype, int *ex, int *ey, int *ez) {
    const int lay = grid_layout(dtype);
    *ex = cow::kBrick + (lay == cow::kLayNat ? 1 : 0);
    *ey = cow::kBrick + (lay == cow::kLayQuad8 ? 0 : 1);
    *ez = cow::kBrick + 1;
}

// smallest e with amax <= 448 * 2^e (e = 0 for an all-zero channel)
int fp8_exponent(float amax) {
    if (!(amax > 0.0f)) return 0;
    int e = 0;
    while ((double)amax > std::ldexp(448.0, e)) e++;
    while ((double)amax <= std::ldexp(448.0, e - 1) && e > -120) e--;
    return e;
}

}  // namespace

namespace {

void destroy(cow_ctx *c) {
    if (!c) return;
    DeviceGuard g(c->device);
    for (cow_batch *b : c->batches) batch_detach(b);  // batches freed later no longer reach the context
    // under a residency budget, calls return with loads from the pinned host
    // copies still queued: let them finish first
    if (c->pool) cudaDeviceSynchronize();
    for (auto &b : c->blocks) {
        if (b.chunk) {  // pool memory: freed in stream order before the pool goes
            cudaFreeAsync(b.chunk, nullptr);
        } else {
            cudaFree(b.grid);
            for (auto *p : b.planes) cudaFree(p);
        }
        b.use_ev.reset();
        cudaFree(b.occ);
        cudaFree(b.occ2);
        cudaFree(b.scale);
        cudaFree(b.brick_tab);
        cudaFree(b.brick_list);
        if (b.host_feat) cudaFreeHost(b.host_feat);
    }
    c->last_call_ev.reset();
    if (c->loaded) cudaEventDestroy(c->loaded);
    if (c->copy_stream) cudaStreamDestroy(c->copy_stream);
    cudaFree(c->d_err);
    cudaFree(c->d_mlp);
    if (c->pool) {
        cudaDeviceSynchronize();  // frees of pool memory queued in stream order have run
        cudaMemPoolDestroy(c->pool);
    }
    c->views.release();
    c->out_rgb.release();
    c->out_aux.release();
    c->out_nsamp.release();
    c->gptrs.release();
    c->f64ptrs.release();
    c->partials.release();
    c->staging.release();
    c->block_mlps.release();
    c->bm_scratch.release();
    c->ray_keys.release();
    c->ray_hist.release();
    c->ray_perm.release();
    delete c;
}


// height of the highest occupied part of a block
double block_ztop(const BlockHost &b, const std::vector<uint32_t> &bits, int C) {
    const int Nc = (b.R - 1 + C - 1) / C;
    for (int cz = Nc - 1; cz >= 0; cz--) {
        for (int64_t k = (int64_t)cz * Nc * Nc; k < (int64_t)(cz + 1) * Nc * Nc; k++) {
            if ((bits[k >> 5] >> (k & 31)) & 1u) {
                int top = std::min((cz + 1) * C, b.R - 1);
                return (double)b.lo[2] + ((double)top * ((double)b.hi[2] - (double)b.lo[2])) / (double)(b.R - 1);
            }
        }
    }
    return (double)b.lo[2];
}

// After the occupancy kernel: z_top, the coarse occupancy level (the OR
// over each group of kOccGroup^3 cells, clipped at the far faces) and, for a
// brick-sparse context, the brick table (a brick is one coarse cell; it is
// stored when its coarse bit is set).
cow_status build_occupancy_levels(cow_ctx *c, BlockHost &b, int Nc, cudaStream_t st) {
    std::vector<uint32_t> bits((size_t)b.occ_words);
    COW_CUDA(cudaMemcpyAsync(bits.data(), b.occ, (size_t)b.occ_words * 4, cudaMemcpyDeviceToHost, st));
    COW_CUDA(cudaStreamSynchronize(st));
    b.ztop = block_ztop(b, bits, c->occ_cell);
    const int Nc2 = (Nc + cow::kOccGroup - 1) / cow::kOccGroup;
    std::vector<uint32_t> coarse(((size_t)Nc2 * Nc2 * Nc2 + 31) / 32, 0u);
    for (int z = 0; z < Nc; z++)
        for (int y = 0; y < Nc; y++)
            for (int x = 0; x < Nc; x++) {
                const int64_t ci = ((int64_t)z * Nc + y) * Nc + x;
                if (!((bits[(size_t)(ci >> 5)] >> (ci & 31)) & 1u)) continue;
                const int64_t c2 = ((int64_t)(z >> cow::kOccGroupLog2) * Nc2 + (y >> cow::kOccGroupLog2)) * Nc2 +
                                   (x >> cow::kOccGroupLog2);
                coarse[(size_t)(c2 >> 5)] |= 1u << (c2 & 31);
            }
    b.occ2_words = (int64_t)coarse.size();
    COW_CUDA(cudaMalloc((void **)&b.occ2, coarse.size() * 4));
    COW_CUDA(cudaMemcpy(b.occ2, coarse.data(), coarse.size() * 4, cudaMemcpyHostToDevice));
    if (!c->bricks) return COW_OK;
    // brick = coarse cell: kOccGroup cells of occ_cell (= 4) voxels = kBrick voxels
    const int nb = Nc2;
    std::vector<int32_t> tab((size_t)nb * nb * nb, -1), list;
    for (int64_t k = 0; k < (int64_t)nb * nb * nb; k++)
        if ((coarse[(size_t)(k >> 5)] >> (k & 31)) & 1u) {
            tab[(size_t)k] = (int32_t)list.size();
            list.push_back((int32_t)k);
        }
    b.Nb = nb;
    b.n_bricks = (int32_t)list.size();
    COW_CUDA(cudaMalloc((void **)&b.brick_tab, tab.size() * 4));
    COW_CUDA(cudaMemcpy(b.brick_tab, tab.data(), tab.size() * 4, cudaMemcpyHostToDevice));
    COW_CUDA(cudaMalloc((void **)&b.brick_list, std::max<size_t>(list.size(), 1) * 4));
    if (!list.empty()) COW_CUDA(cudaMemcpy(b.brick_list, list.data(), list.size() * 4, cudaMemcpyHostToDevice));
    return COW_OK;
}

// Elements of a block's packed grid: dense R^3, or its stored bricks; and
// (FP8 with BF16 density) of the density octets that follow them.
int64_t grid_elems(const cow_ctx *c, const BlockHost &b) {
    if (b.Nb == 0) return (int64_t)b.R * b.R * b.R;
    int ex, ey, ez;
    brick_dims(c->dtype, &ex, &ey, &ez);
    return (int64_t)b.n_bricks * ex * ey * ez;
}
int64_t dens_elems(const cow_ctx *c, const BlockHost &b) {
    if (c->dtype != COW_FP8_BF16D) return 0;
    return b.Nb == 0 ? (int64_t)b.R * b.R * b.R : (int64_t)b.n_bricks * cow::kDensBrickElems;
}
int64_t grid_main_bytes(const cow_ctx *c, const BlockHost &b) { return grid_elems(c, b) * packed_elem_bytes(c->dtype); }

// Pack the grid master s (device, R^3 x 8) into b.grid (and its density
// octets); d_inv: the grid's 8 inverse channel scales (device).
cow_status pack_grid(cow_ctx *c, BlockHost &b, const float *s, const float *d_inv, cudaStream_t st) {
    const int R = b.R;
    if (b.Nb == 0 && c->dtype != COW_FP8_BF16D) {
        COW_CUDA(cow::launch_pack(s, (int64_t)R * R * R, R, tensor_dtype(c->dtype, 0), d_inv, b.grid, st));
        return COW_OK;
    }
    int ex, ey, ez;
    brick_dims(c->dtype, &ex, &ey, &ez);
    const bool sparse = b.Nb > 0;
    const int sy = sparse ? ex : R, sz = sparse ? ex * ey : R * R, belem = sparse ? ex * ey * ez : 0;
    COW_CUDA(cow::launch_pack_grid(s, R, grid_elems(c, b), sy, sz, belem, sparse ? b.brick_list : nullptr, b.Nb,
                                   tensor_dtype(c->dtype, 0), grid_layout(c->dtype), d_inv, b.grid, st));
    if (c->dtype == COW_FP8_BF16D) {
        void *dens = (unsigned char *)b.grid + grid_main_bytes(c, b);
        const int dsy = sparse ? cow::kBrick : R, dsz = sparse ? cow::kBrick * cow::kBrick : R * R;
        COW_CUDA(cow::launch_pack_grid(s, R, dens_elems(c, b), dsy, dsz, sparse ? cow::kDensBrickElems : 0,
                                       sparse ? b.brick_list : nullptr, b.Nb, COW_BF16, cow::kLayOct16, nullptr, dens,
                                       st));
    }
    return COW_OK;
}

// FP8 scale exponents of one tensor (8 channels) from its device master:
// e[k] = 0 unless the tensor is stored in FP8.
cow_status fp8_exponents(const cow_ctx *c, int t, const float *s, int64_t nv, unsigned *d_amax, cudaStream_t st,
                         int e[8]) {
    for (int k = 0; k < 8; k++) e[k] = 0;
    if (tensor_dtype(c->dtype, t) != COW_FP8_E4M3) return COW_OK;
    COW_CUDA(cow::launch_amax8(s, nv, d_amax, st));
    unsigned amax_bits[8];
    COW_CUDA(cudaMemcpyAsync(amax_bits, d_amax, sizeof(amax_bits), cudaMemcpyDeviceToHost, st));
    COW_CUDA(cudaStreamSynchronize(st));
    for (int k = 0; k < 8; k++) {
        float a;
        std::memcpy(&a, &amax_bits[k], 4);
        e[k] = fp8_exponent(a);
    }
    return COW_OK;
}

// Pack tensor t of block b from its device master s (grid or plane).
cow_status pack_tensor(cow_ctx *c, BlockHost &b, int t, const float *s, const float *d_inv, cudaStream_t st) {
    if (t == 0) return pack_grid(c, b, s, d_inv, st);
    if (c->dtype == COW_BF16_FP8 || c->dtype == COW_FP8_BF16D)
        COW_CUDA(cow::launch_pack_quad8(s, b.P, d_inv, b.planes[t - 1], st));
    else
        COW_CUDA(cow::launch_pack(s, (int64_t)b.P * b.P, b.P, tensor_dtype(c->dtype, t), d_inv, b.planes[t - 1], st));
    return COW_OK;
}

// Re-pack the features of an existing block from new FP32 masters (occupancy,
// z_top and the brick set unchanged); FP8 scales are recomputed.
cow_status repack_block(cow_ctx *c, BlockHost &b, const float *const src_in[4], void *staging, unsigned *d_amax,
                        float *d_inv, cudaStream_t st) {
    const int64_t nv[4] = {(int64_t)b.R * b.R * b.R, (int64_t)b.P * b.P, (int64_t)b.P * b.P, (int64_t)b.P * b.P};
    float scale_h[32];
    for (int t = 0; t < 4; t++) {
        const float *s = src_in[t];
        if (!is_device_ptr(s)) {
            COW_CUDA(cudaMemcpyAsync(staging, s, (size_t)nv[t] * 32, cudaMemcpyHostToDevice, st));
            s = (const float *)staging;
        }
        int e[8];
        cow_status rc = fp8_exponents(c, t, s, nv[t], d_amax, st, e);
        if (rc != COW_OK) return rc;
        float inv[8];
        for (int k = 0; k < 8; k++) {
            b.scale_exp[t][k] = e[k];
            inv[k] = std::ldexp(1.0f, -e[k]);
            scale_h[8 * t + k] = std::ldexp(1.0f, e[k]);
        }
        COW_CUDA(cudaMemcpyAsync(d_inv + 8 * t, inv, sizeof(inv), cudaMemcpyHostToDevice, st));
        if ((rc = pack_tensor(c, b, t, s, d_inv + 8 * t, st)) != COW_OK) return rc;
    }
    COW_CUDA(cudaMemcpyAsync(b.scale, scale_h, sizeof(scale_h), cudaMemcpyHostToDevice, st));
    return COW_OK;
}

cow_status load_one(cow_ctx *c, const cow_block_desc &d, BlockHost &b, void *staging, unsigned *d_amax,
                    float *d_inv, double log_thresh, cudaStream_t st) {
    const int64_t nv[4] = {(int64_t)d.grid_res * d.grid_res * d.grid_res, (int64_t)d.plane_res * d.plane_res,
                           (int64_t)d.plane_res * d.plane_res, (int64_t)d.plane_res * d.plane_res};
    const float *src[4] = {d.grid, d.planes[0], d.planes[1], d.planes[2]};
    const int Nc = (d.grid_res - 1 + c->occ_cell - 1) / c->occ_cell;
    b.occ_words = ((int64_t)Nc * Nc * Nc + 31) / 32;
    COW_CUDA(cudaMalloc((void **)&b.occ, (size_t)b.occ_words * 4));
    COW_CUDA(cudaMalloc((void **)&b.scale, 32 * sizeof(float)));
    float scale_h[32];
    // the grid first: its occupancy decides the coarse level and, for a
    // brick-sparse grid, which bricks are stored
    for (int t = 0; t < 4; t++) {
        const float *s = src[t];
        if (!is_device_ptr(s)) {
            COW_CUDA(cudaMemcpyAsync(staging, s, (size_t)nv[t] * 32, cudaMemcpyHostToDevice, st));
            s = (const float *)staging;
        }
        int e[8];
        cow_status rc = fp8_exponents(c, t, s, nv[t], d_amax, st, e);
        if (rc != COW_OK) return rc;
        float inv[8];
        for (int k = 0; k < 8; k++) {
            b.scale_exp[t][k] = e[k];
            inv[k] = std::ldexp(1.0f, -e[k]);
            scale_h[8 * t + k] = std::ldexp(1.0f, e[k]);
        }
        COW_CUDA(cudaMemcpyAsync(d_inv, inv, sizeof(inv), cudaMemcpyHostToDevice, st));
        if (t == 0) {
            COW_CUDA(cow::launch_occupancy(s, d.grid_res, c->occ_cell, log_thresh, b.occ, st));
            if ((rc = build_occupancy_levels(c, b, Nc, st)) != COW_OK) return rc;
            COW_CUDA(cudaMalloc(&b.grid, (size_t)(grid_main_bytes(c, b) + dens_elems(c, b) * 16)));
        } else {
            COW_CUDA(cudaMalloc(&b.planes[t - 1], (size_t)(nv[t] * packed_elem_bytes(c->dtype))));
        }
        if ((rc = pack_tensor(c, b, t, s, d_inv, st)) != COW_OK) return rc;
        // the staging buffer and d_inv are reused by the next tensor: the
        // stream orders the next copies after these kernels
    }
    COW_CUDA(cudaMemcpyAsync(b.scale, scale_h, sizeof(scale_h), cudaMemcpyHostToDevice, st));
    return COW_OK;
}

cow::BlockRec make_rec(const cow_ctx *c, const BlockHost &b) {
    cow::BlockRec r;
    std::memset(&r, 0, sizeof(r));
    for (int a = 0; a < 3; a++) {
        r.lo[a] = b.lo[a];
        r.hi[a] = b.hi[a];
        const double ext = (double)b.hi[a] - (double)b.lo[a];
        const double m = 1e-3 * std::max(1.0, ext);
        r.lo_e[a] = (float)((double)b.lo[a] - m);
        r.hi_e[a] = (float)((double)b.hi[a] + m);
        r.kg[a] = (float)((double)(b.R - 1) / ext);
        r.kp[a] = (float)((double)(b.P - 1) / ext);
    }
    r.delta = (float)(((double)b.hi[0] - (double)b.lo[0]) / (double)b.P);
    double bm = 0.0;
    for (int a = 0; a < 3; a++) {
        r.vox[a] = (float)(((double)b.hi[a] - (double)b.lo[a]) / (double)(b.R - 1));
        bm = std::max(bm, std::max(std::fabs((double)b.lo[a]), std::fabs((double)b.hi[a])));
    }
    r.bmax = (float)bm;
    r.cx = (float)(0.5 * ((double)b.lo[0] + (double)b.hi[0]));
    r.cy = (float)(0.5 * ((double)b.lo[1] + (double)b.hi[1]));
    r.R = b.R;
    r.P = b.P;
    r.C = c->occ_cell;
    r.Nc = (b.R - 1 + c->occ_cell - 1) / c->occ_cell;
    r.cdiv = c->occ_cell > 1 ? (uint32_t)((0x100000000ull + (uint64_t)c->occ_cell - 1) / (uint64_t)c->occ_cell) : 0u;
    r.dtype = c->dtype;
    r.grid = b.grid;
    r.dens = (b.grid && c->dtype == COW_FP8_BF16D) ? (const unsigned char *)b.grid + grid_main_bytes(c, b) : nullptr;
    if (b.Nb > 0) {
        int ex, ey, ez;
        brick_dims(c->dtype, &ex, &ey, &ez);
        r.brick = b.brick_tab;
        r.Nb = b.Nb;
        r.bsy = ex;
        r.bsz = ex * ey;
        r.belem = ex * ey * ez;
    } else {
        r.brick = nullptr;
        r.Nb = 0;
        r.bsy = b.R;
        r.bsz = b.R * b.R;
        r.belem = 0;
    }
    for (int k = 0; k < 3; k++) r.planes[k] = b.planes[k];
    r.occ = b.occ;
    r.scale = b.scale;
    r.occ2 = b.occ2;
    r.Nc2 = (r.Nc + cow::kOccGroup - 1) / cow::kOccGroup;
    r.unb = b.unb;
    for (int a = 0; a < 3; a++) {
        r.cc[a] = (float)(0.5 * ((double)b.lo[a] + (double)b.hi[a]));
        r.ih[a] = (float)(2.0 / ((double)b.hi[a] - (double)b.lo[a]));
        r.plo[a] = r.lo[a];
    }
    if (b.unb & cow::kUnbContracted) {
        // lookups index the contracted coordinate u in [-2, 2]
        for (int a = 0; a < 3; a++) {
            r.plo[a] = -2.0f;
            r.kg[a] = (float)((double)(b.R - 1) / 4.0);
            r.kp[a] = (float)((double)(b.P - 1) / 4.0);
        }
    }
    return r;
}

// --- App. D on the host, FP64 ---------------------------------------------

struct ViewGeom {
    double t[3];
    double m[9];  // rotation, row-major
    double kx, ky;
};

ViewGeom view_geom(const cow_camera &cam) {
    ViewGeom g;
    for (int r = 0; r < 3; r++) {
        g.t[r] = cam.c2w[4 * r + 3];
        for (int k = 0; k < 3; k++) g.m[3 * r + k] = cam.c2w[4 * r + k];
    }
    const double f = focal_length(cam.height, cam.fov_y_deg);
    g.kx = (double)cam.width / (2.0 * f);
    g.ky = (double)cam.height / (2.0 * f);
    return g;
}

// Conservative: culled only when all 8 corners are strictly outside one plane.
bool box_in_view(const ViewGeom &g, const double lo[3], const double hi[3]) {
    bool all_out[5] = {true, true, true, true, true};
    for (int k = 0; k < 8; k++) {
        const double q0 = ((k & 1) ? hi[0] : lo[0]) - g.t[0];
        const double q1 = ((k & 2) ? hi[1] : lo[1]) - g.t[1];
        const double q2 = ((k & 4) ? hi[2] : lo[2]) - g.t[2];
        // camera-frame coordinates: transpose(rotation) * q
        const double xc = (g.m[0] * q0 + g.m[3] * q1) + g.m[6] * q2;
        const double yc = (g.m[1] * q0 + g.m[4] * q1) + g.m[7] * q2;
        const double zc = (g.m[2] * q0 + g.m[5] * q1) + g.m[8] * q2;
        const double depth = -zc;
        const double side[5] = {depth, xc + g.kx * depth, g.kx * depth - xc, yc + g.ky * depth, g.ky * depth - yc};
        for (int s = 0; s < 5; s++) all_out[s] = all_out[s] && (side[s] < 0.0);
    }
    return !(all_out[0] || all_out[1] || all_out[2] || all_out[3] || all_out[4]);
}

bool block_in_view(const ViewGeom &g, const BlockHost &b) {
    const double lo[3] = {b.lo[0], b.lo[1], b.lo[2]};
    const double hi[3] = {b.hi[0], b.hi[1], b.ztop};
    return box_in_view(g, lo, hi);
}

double block_range(const ViewGeom &g, const BlockHost &b) {
    const double dx = 0.5 * ((double)b.lo[0] + (double)b.hi[0]) - g.t[0];
    const double dy = 0.5 * ((double)b.lo[1] + (double)b.hi[1]) - g.t[1];
    const double dz = b.ztop - g.t[2];
    return std::sqrt((dx * dx + dy * dy) + dz * dz);
}

void depth_sort(const cow_ctx *c, const cow_camera &cam, std::vector<int32_t> &ids) {
    std::vector<std::pair<double, int32_t>> keyed;
    keyed.reserve(ids.size());
    for (int32_t id : ids) {
        const BlockHost &b = c->blocks[id];
        const double dx = 0.5 * ((double)b.lo[0] + (double)b.hi[0]) - cam.c2w[3];
        const double dy = 0.5 * ((double)b.lo[1] + (double)b.hi[1]) - cam.c2w[7];
        keyed.emplace_back(dx * dx + dy * dy, id);
    }
    std::sort(keyed.begin(), keyed.end());  // (key, id): ties by index
    for (size_t k = 0; k < ids.size(); k++) ids[k] = keyed[k].second;
}

// Sizes one launch processes; shared by cow_render and its host-output path.
struct ViewPlan {
    std::vector<cow::ViewRec> recs;
    int64_t n_pix = 0;
    int n_tiles = 0;
};

cow_status plan_views(const cow_ctx *c, const cow_camera *cams, int32_t n_views, const int32_t *ids,
                      const int32_t *ids_offsets, ViewPlan &plan) {
    const int tw = cow::march_tile_w(), th = cow::march_tile_h();
    plan.recs.resize((size_t)n_views);
    int64_t tiles = 0;
    const int32_t nb = (int32_t)c->blocks.size();
    if (ids_offsets[0] != 0) return fail(COW_ERR_INVALID_ARG, "ids_offsets[0] must be 0");
    for (int32_t v = 0; v < n_views; v++) {
        const cow_camera &cam = cams[v];
        if (cam.width < 1 || cam.height < 1 || cam.width > 32768 || cam.height > 32768)
            return fail(COW_ERR_INVALID_ARG, "view %d: bad image size %dx%d", v, cam.width, cam.height);
        if (!(cam.fov_y_deg > 0.0 && cam.fov_y_deg < 180.0))
            return fail(COW_ERR_INVALID_ARG, "view %d: fov_y_deg must be in (0, 180)", v);
        if (ids_offsets[v + 1] < ids_offsets[v])
            return fail(COW_ERR_INVALID_ARG, "ids_offsets must be non-decreasing");
        for (int32_t k = ids_offsets[v]; k < ids_offsets[v + 1]; k++)
            if (ids[k] < 0 || ids[k] >= nb) return fail(COW_ERR_INVALID_ARG, "view %d: block id %d out of range", v, ids[k]);
        cow::ViewRec &r = plan.recs[(size_t)v];
        std::memset(&r, 0, sizeof(r));
        for (int rr = 0; rr < 3; rr++) {
            for (int k = 0; k < 3; k++) r.Rm[3 * rr + k] = (float)cam.c2w[4 * rr + k];
            r.o[rr] = (float)cam.c2w[4 * rr + 3];
        }
        r.f = (float)focal_length(cam.height, cam.fov_y_deg);
        r.W = cam.width;
        r.H = cam.height;
        r.tiles_x = (cam.width + tw - 1) / tw;
        const int tiles_y = (cam.height + th - 1) / th;
        r.tile_begin = (int32_t)tiles;
        r.ids_begin = ids_offsets[v];
        r.ids_count = ids_offsets[v + 1] - ids_offsets[v];
        r.strip = c->tile_strip;
        r.pix_offset = plan.n_pix;
        tiles += (int64_t)r.tiles_x * tiles_y;
        plan.n_pix += (int64_t)cam.width * cam.height;
    }
    if (tiles > 0x7fffffff) return fail(COW_ERR_INVALID_ARG, "too many tiles in one call");
    plan.n_tiles = (int)tiles;
    return COW_OK;
}

// Resolve an output pointer: device memory is used in place, host memory goes
// through a context buffer copied back after the kernel.
template <typename T>
cow_status resolve_out(T *user, size_t bytes, DevBuf &buf, T **dev, bool *host) {
    *host = false;
    *dev = user;
    if (!user) return COW_OK;
    if (is_device_ptr(user)) return COW_OK;
    // page-locked host memory mapped into the device's address space (on a
    // Grace-Blackwell node, reached over the coherent chip-to-chip link):
    // the kernel writes the outputs there directly, spread over its run,
    // instead of a copy of the whole frame after it
    cudaPointerAttributes at;
    if (cudaPointerGetAttributes(&at, user) == cudaSuccess && at.type == cudaMemoryTypeHost && at.devicePointer) {
        *dev = (T *)at.devicePointer;
        return COW_OK;
    }
    cudaGetLastError();
    COW_CUDA(buf.reserve(bytes));
    *dev = (T *)buf.p;
    *host = true;
    return COW_OK;
}

cow_status resolve_mlp(cow_ctx *c, const float *mlp, cudaStream_t st, const float **dev) {
    if (is_device_ptr(mlp)) {
        *dev = mlp;
        return COW_OK;
    }
    COW_CUDA(cudaMemcpyAsync(c->d_mlp, mlp, cow::kMlpParams * sizeof(float), cudaMemcpyHostToDevice, st));
    *dev = c->d_mlp;
    return COW_OK;
}

// The records of a ray-batch call's blocks, for the launch's parameter buffer
// (call after the blocks are loaded: the records carry their pointers).
void make_ray_recs(const cow_ctx *c, const int32_t *ids, int32_t n, cow::RayRecs &rr) {
    std::memset(&rr, 0, sizeof(rr));
    rr.n = n;
    for (int32_t k = 0; k < n; k++) {
        rr.r[k] = c->recs[(size_t)ids[k]];
        rr.id[k] = ids[k];
    }
}

// The coherent processing order of a ray batch (cow_set_ray_order), or null
// for the order given: batches below kRayOrderMin rays keep theirs (the sort
// would cost more than it saves).  The box is the call's blocks' bounding
// box.  The permutation lives in the context until the next call.
constexpr int64_t kRayOrderMin = 8192;

cow_status ray_order(cow_ctx *c, const float *o, const float *d, int64_t n, const int32_t *ids, int32_t n_ids,
                     cudaStream_t st, const int32_t **perm) {
    *perm = nullptr;
    if (c->ray_order != COW_RAY_ORDER_COHERENT || n < kRayOrderMin || n > 0x7fffffff) return COW_OK;
    float lo[3] = {3.0e38f, 3.0e38f, 3.0e38f}, hi[3] = {-3.0e38f, -3.0e38f, -3.0e38f};
    for (int32_t k = 0; k < n_ids; k++) {
        const BlockHost &b = c->blocks[(size_t)ids[k]];
        for (int a = 0; a < 3; a++) {
            lo[a] = std::min(lo[a], b.lo[a]);
            hi[a] = std::max(hi[a], b.hi[a]);
        }
    }
    COW_CUDA(c->ray_keys.reserve((size_t)n * sizeof(uint32_t)));
    COW_CUDA(c->ray_hist.reserve((size_t)cow::kRayOrderHistWords * sizeof(uint32_t)));
    COW_CUDA(c->ray_perm.reserve((size_t)n * sizeof(int32_t)));
    COW_CUDA(cow::launch_ray_order(o, d, n, lo, hi, (uint32_t *)c->ray_keys.p, (uint32_t *)c->ray_hist.p,
                                   (int32_t *)c->ray_perm.p, st));
    *perm = (const int32_t *)c->ray_perm.p;
    return COW_OK;
}

// --- dynamic loading / unloading under a device-memory budget (App. D) -----
// The packed grid and planes of a block are its loadable resources; the
// occupancy levels, scales and records stay resident (a few KB per block).

int64_t tensor_bytes(const cow_ctx *c, const BlockHost &b, int t) {
    if (t == 0) return grid_main_bytes(c, b) + dens_elems(c, b) * 16;
    return (int64_t)b.P * b.P * packed_elem_bytes(c->dtype);
}

int64_t feature_bytes(const cow_ctx *c, const BlockHost &b) {
    int64_t s = 0;
    for (int t = 0; t < 4; t++) s += tensor_bytes(c, b, t);
    return s;
}

void **tensor_slot(BlockHost &b, int t) { return t == 0 ? &b.grid : &b.planes[t - 1]; }

// Offset of tensor t in a block's host copy and pooled chunk (256-byte
// aligned), and the chunk's size.
int64_t feature_offset(const cow_ctx *c, const BlockHost &b, int t) {
    int64_t off = 0;
    for (int u = 0; u < t; u++) off = (off + tensor_bytes(c, b, u) + 255) & ~(int64_t)255;
    return off;
}
int64_t chunk_bytes(const cow_ctx *c, const BlockHost &b) { return feature_offset(c, b, 3) + tensor_bytes(c, b, 3); }

// Rewrite the host record of block i.  Kernels receive records by value (in
// their parameter buffer or a per-call staging copy), so no device table
// needs the change and the host does not wait for the stream.
cow_status refresh_rec(cow_ctx *c, int32_t i, cudaStream_t) {
    c->recs[(size_t)i] = make_rec(c, c->blocks[(size_t)i]);
    c->rec_gen++;
    return COW_OK;
}

// Unload block i on the copy stream, after the kernels that read it: write a
// changed device copy back to the host copy, then free the device memory.
cow_status evict_block(cow_ctx *c, int32_t i) {
    BlockHost &b = c->blocks[(size_t)i];
    if (!b.resident) return COW_OK;
    cudaStream_t cs = c->copy_stream;
    if (b.use_ev) {
        COW_CUDA(cudaStreamWaitEvent(cs, b.use_ev->e, 0));
        if (b.use_ev == c->last_call_ev) c->n_evict_wait_last++;
    }
    if (b.dirty) {  // features changed on the device since the host copy was taken
        for (int t = 0; t < 4; t++)
            COW_CUDA(cudaMemcpyAsync((unsigned char *)b.host_feat + feature_offset(c, b, t), *tensor_slot(b, t),
                                     (size_t)tensor_bytes(c, b, t), cudaMemcpyDeviceToHost, cs));
        b.dirty = false;
    }
    if (b.chunk) {
        // back to the pool in the copy stream's order: the next loads reuse it
        COW_CUDA(cudaFreeAsync(b.chunk, cs));
    } else {
        // the load-time allocations: freed once the copy stream has passed
        // the kernels that read them (and the write-back)
        COW_CUDA(cudaStreamSynchronize(cs));
        for (int t = 0; t < 4; t++) COW_CUDA(cudaFree(*tensor_slot(b, t)));
    }
    b.chunk = nullptr;
    for (int t = 0; t < 4; t++) *tensor_slot(b, t) = nullptr;
    b.use_ev.reset();
    b.resident = false;
    c->resident_bytes -= feature_bytes(c, b);
    c->n_evictions++;
    return refresh_rec(c, i, cs);
}

// Load block i on the copy stream: one chunk from the pool, one copy.
cow_status upload_block(cow_ctx *c, int32_t i) {
    BlockHost &b = c->blocks[(size_t)i];
    if (b.resident) return COW_OK;
    cudaStream_t cs = c->copy_stream;
    void *chunk = nullptr;
    const cudaError_t e = cudaMallocFromPoolAsync(&chunk, (size_t)chunk_bytes(c, b), c->pool, cs);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return fail(e == cudaErrorMemoryAllocation ? COW_ERR_OOM : COW_ERR_CUDA, "loading block %d: %s", i,
                    cudaGetErrorString(e));
    }
    COW_CUDA(cudaMemcpyAsync(chunk, b.host_feat, (size_t)chunk_bytes(c, b), cudaMemcpyHostToDevice, cs));
    b.chunk = chunk;
    for (int t = 0; t < 4; t++) *tensor_slot(b, t) = (unsigned char *)chunk + feature_offset(c, b, t);
    b.resident = true;
    const int64_t bytes = feature_bytes(c, b);
    c->resident_bytes += bytes;
    c->n_uploads++;
    c->upload_bytes += bytes;
    return refresh_rec(c, i, cs);
}

// Make the blocks of one call resident: unload the least recently used
// blocks the call does not need until the missing ones fit the budget, then
// load those (in id order).  Loads and unloads go to the copy stream; st
// waits for the loads.
cow_status ensure_resident(cow_ctx *c, const int32_t *ids, int64_t n, cudaStream_t st) {
    if (c->budget <= 0) return COW_OK;
    const int32_t nb = (int32_t)c->blocks.size();
    std::vector<char> need((size_t)nb, 0);
    for (int64_t k = 0; k < n; k++) need[(size_t)ids[k]] = 1;
    int64_t need_bytes = 0, missing = 0;
    for (int32_t i = 0; i < nb; i++)
        if (need[(size_t)i]) {
            const int64_t by = feature_bytes(c, c->blocks[(size_t)i]);
            need_bytes += by;
            if (!c->blocks[(size_t)i].resident) missing += by;
        }
    if (need_bytes > c->budget)
        return fail(COW_ERR_OOM, "the call's blocks need %lld bytes, over the residency budget of %lld",
                    (long long)need_bytes, (long long)c->budget);
    const uint64_t now = ++c->use_clock;
    for (int32_t i = 0; i < nb; i++)
        if (need[(size_t)i]) c->blocks[(size_t)i].last_use = now;
    while (c->resident_bytes + missing > c->budget) {
        int32_t victim = -1;
        for (int32_t i = 0; i < nb; i++) {
            const BlockHost &b = c->blocks[(size_t)i];
            if (!b.resident || need[(size_t)i]) continue;
            if (victim < 0 || b.last_use < c->blocks[(size_t)victim].last_use) victim = i;
        }
        if (victim < 0) break;  // cannot happen: the needed blocks alone fit
        cow_status rc = evict_block(c, victim);
        if (rc != COW_OK) return rc;
    }
    bool loaded = false;
    for (int32_t i = 0; i < nb; i++)
        if (need[(size_t)i] && !c->blocks[(size_t)i].resident) {
            cow_status rc = upload_block(c, i);
            if (rc != COW_OK) return rc;
            loaded = true;
        }
    if (loaded) {
        COW_CUDA(cudaEventRecord(c->loaded, c->copy_stream));
        COW_CUDA(cudaStreamWaitEvent(st, c->loaded, 0));
    }
    return COW_OK;
}

cow_status note_use_impl(cow_ctx *c, const int32_t *ids, int64_t n, cudaStream_t st) {
    if (c->budget <= 0 || n <= 0) return COW_OK;
    auto ev = std::make_shared<SharedEvent>();
    if (!ev->e) return fail(COW_ERR_CUDA, "cudaEventCreate failed");
    COW_CUDA(cudaEventRecord(ev->e, st));
    for (int64_t k = 0; k < n; k++) c->blocks[(size_t)ids[k]].use_ev = ev;
    c->last_call_ev = ev;
    return COW_OK;
}

}  // namespace

namespace cowi {

int64_t block_feature_bytes(const cow_ctx *c, int32_t i) { return feature_bytes(c, c->blocks[(size_t)i]); }

cow_status make_resident(cow_ctx *c, const int32_t *ids, int64_t n, cudaStream_t st) {
    return ensure_resident(c, ids, n, st);
}

cow_status note_use(cow_ctx *c, const int32_t *ids, int64_t n, cudaStream_t st) {
    return note_use_impl(c, ids, n, st);
}

int64_t block_tensor_bytes(const cow_ctx *c, const BlockHost &b, int t) { return tensor_bytes(c, b, t); }
int64_t block_feature_offset(const cow_ctx *c, const BlockHost &b, int t) { return feature_offset(c, b, t); }
cow::BlockRec block_record(const cow_ctx *c, const BlockHost &b) { return make_rec(c, b); }
void destroy_context(cow_ctx *c) { destroy(c); }

}  // namespace cowi

extern "C" {

int32_t cow_version(void) { return 1; }

const char *cow_last_error(void) { return g_last_error.c_str(); }

cow_status cow_load_blocks(cow_ctx **out, const cow_block_desc *blocks, int32_t n, cow_dtype storage,
                           float occ_thresh, int32_t occ_cell, void *stream) {
    return cow_load_blocks_ex(out, blocks, n, storage, occ_thresh, occ_cell, 0u, stream);
}

cow_status cow_load_blocks_ex(cow_ctx **out, const cow_block_desc *blocks, int32_t n, cow_dtype storage,
                              float occ_thresh, int32_t occ_cell, uint32_t load_flags, void *stream) {
    COW_NVTX("cow_load_blocks_ex");
    g_last_error.clear();
    if (!out || !blocks || n < 1) return fail(COW_ERR_INVALID_ARG, "cow_load_blocks: null pointer or n < 1");
    *out = nullptr;
    if ((int)storage < 0 || (int)storage > 5) return fail(COW_ERR_INVALID_ARG, "unknown storage dtype %d", (int)storage);
    if (load_flags & ~(uint32_t)COW_LOAD_BRICKS) return fail(COW_ERR_INVALID_ARG, "unknown load flags 0x%x", load_flags);
    if (occ_cell < 1 || occ_cell > 4096) return fail(COW_ERR_INVALID_ARG, "occ_cell must be in [1, 4096]");
    if ((load_flags & COW_LOAD_BRICKS) && occ_cell != 4)
        return fail(COW_ERR_UNSUPPORTED, "brick-sparse grids need occ_cell = 4 (a brick is 4 x 4 cells of 4 voxels)");
    if (!(occ_thresh > 0.0f)) return fail(COW_ERR_INVALID_ARG, "occ_thresh must be > 0");
    size_t max_vec = 0;
    for (int32_t i = 0; i < n; i++) {
        const cow_block_desc &d = blocks[i];
        if (!d.grid || !d.planes[0] || !d.planes[1] || !d.planes[2])
            return fail(COW_ERR_INVALID_ARG, "block %d: null array", i);
        for (const float *q : {d.grid, d.planes[0], d.planes[1], d.planes[2]})
            if (((uintptr_t)q & 15u) != 0) return fail(COW_ERR_INVALID_ARG, "block %d: arrays must be 16-byte aligned", i);
        if (d.grid_res < 2 || d.plane_res < 2 || d.grid_res > 1024 || d.plane_res > 16384)
            return fail(COW_ERR_INVALID_ARG, "block %d: resolutions must be in [2, 1024] / [2, 16384]", i);
        for (int a = 0; a < 3; a++)
            if (!(d.lo[a] < d.hi[a])) return fail(COW_ERR_INVALID_ARG, "block %d: lo must be < hi", i);
        if (d.lod < 1) return fail(COW_ERR_INVALID_ARG, "block %d: lod must be >= 1", i);
        if (d.parent < -1 || d.parent >= n || d.parent == i)
            return fail(COW_ERR_INVALID_ARG, "block %d: bad parent index %d", i, d.parent);
        if (d.parent >= 0 && blocks[d.parent].lod != d.lod + 1)
            return fail(COW_ERR_INVALID_ARG, "block %d: parent must be one level coarser", i);
        max_vec = std::max(max_vec, (size_t)d.grid_res * d.grid_res * d.grid_res);
        max_vec = std::max(max_vec, (size_t)d.plane_res * d.plane_res);
    }
    cow_ctx *c = new cow_ctx();
    cudaStream_t st = (cudaStream_t)stream;
    if (cudaGetDevice(&c->device) != cudaSuccess) {
        delete c;
        return fail(COW_ERR_CUDA, "no CUDA device");
    }
    c->dtype = (int)storage;
    c->bricks = (load_flags & COW_LOAD_BRICKS) != 0;
    c->occ_cell = occ_cell;
    c->occ_thresh = occ_thresh;
    c->blocks.resize((size_t)n);
    void *staging = nullptr;
    unsigned *d_amax = nullptr;
    float *d_inv = nullptr;
    cow_status rc = COW_OK;
    auto cleanup = [&](cow_status s) {
        cudaFree(staging);
        cudaFree(d_amax);
        cudaFree(d_inv);
        if (s != COW_OK) destroy(c);
        return s;
    };
    bool any_host = false;
    for (int32_t i = 0; i < n && !any_host; i++) {
        const cow_block_desc &d = blocks[i];
        any_host = !is_device_ptr(d.grid) || !is_device_ptr(d.planes[0]) || !is_device_ptr(d.planes[1]) ||
                   !is_device_ptr(d.planes[2]);
    }
    cudaError_t e = cudaSuccess;
    if (any_host) e = cudaMalloc(&staging, max_vec * 32);
    if (e == cudaSuccess) e = cudaMalloc((void **)&d_amax, 8 * sizeof(unsigned));
    if (e == cudaSuccess) e = cudaMalloc((void **)&d_inv, 8 * sizeof(float));
    if (e == cudaSuccess) e = cudaMalloc((void **)&c->d_err, sizeof(unsigned));
    if (e == cudaSuccess) e = cudaMalloc((void **)&c->d_mlp, 512 * sizeof(float));
    if (e == cudaSuccess) e = cudaMemsetAsync(c->d_err, 0, sizeof(unsigned), st);
    if (e != cudaSuccess)
        return cleanup(fail(e == cudaErrorMemoryAllocation ? COW_ERR_OOM : COW_ERR_CUDA, "cow_load_blocks: %s",
                            cudaGetErrorString(e)));
    const double log_thresh = std::log((double)occ_thresh);
    for (int32_t i = 0; i < n && rc == COW_OK; i++) {
        const cow_block_desc &d = blocks[i];
        BlockHost &b = c->blocks[(size_t)i];
        for (int a = 0; a < 3; a++) {
            b.lo[a] = d.lo[a];
            b.hi[a] = d.hi[a];
        }
        b.lod = d.lod;
        b.parent = d.parent;
        b.R = d.grid_res;
        b.P = d.plane_res;
        rc = load_one(c, d, b, staging, d_amax, d_inv, log_thresh, st);
    }
    if (rc != COW_OK) return cleanup(rc);
    for (int32_t i = 0; i < n; i++)
        if (blocks[i].parent >= 0) c->blocks[(size_t)blocks[i].parent].children.push_back(i);
    std::vector<cow::BlockRec> &recs = c->recs;
    recs.resize((size_t)n);
    for (int32_t i = 0; i < n; i++) recs[(size_t)i] = make_rec(c, c->blocks[(size_t)i]);
    e = cudaStreamSynchronize(st);
    if (e != cudaSuccess)
        return cleanup(fail(e == cudaErrorMemoryAllocation ? COW_ERR_OOM : COW_ERR_CUDA, "cow_load_blocks: %s",
                            cudaGetErrorString(e)));
    cleanup(COW_OK);
    *out = c;
    return COW_OK;
}

cow_status cow_free(cow_ctx *ctx) {
    destroy(ctx);
    return COW_OK;
}

cow_status cow_num_blocks(const cow_ctx *ctx, int32_t *out_n) {
    if (!ctx || !out_n) return fail(COW_ERR_INVALID_ARG, "null argument");
    *out_n = (int32_t)ctx->blocks.size();
    return COW_OK;
}

cow_status cow_block_ztop(const cow_ctx *ctx, int32_t block, double *out_ztop) {
    if (!ctx || !out_ztop) return fail(COW_ERR_INVALID_ARG, "null argument");
    if (block < 0 || block >= (int32_t)ctx->blocks.size()) return fail(COW_ERR_INVALID_ARG, "block out of range");
    *out_ztop = ctx->blocks[(size_t)block].ztop;
    return COW_OK;
}

cow_status cow_select_lod(const cow_ctx *ctx, const cow_camera *cam, const double *lod_thresh, int32_t n_lod,
                          int32_t *out_ids, int32_t cap, int32_t *out_n) {
    COW_NVTX("cow_select_lod");
    if (!ctx || !cam || !out_n || (n_lod > 0 && !lod_thresh) || (cap > 0 && !out_ids))
        return fail(COW_ERR_INVALID_ARG, "cow_select_lod: null argument");
    const ViewGeom g = view_geom(*cam);
    int32_t top = 1;
    for (const auto &b : ctx->blocks) top = std::max(top, b.lod);
    std::vector<int32_t> sel, stack;
    for (int32_t i = (int32_t)ctx->blocks.size() - 1; i >= 0; i--)
        if (ctx->blocks[(size_t)i].lod == top && block_in_view(g, ctx->blocks[(size_t)i])) stack.push_back(i);
    while (!stack.empty()) {
        const int32_t i = stack.back();
        stack.pop_back();
        const BlockHost &b = ctx->blocks[(size_t)i];
        if (b.lod <= 1) {
            sel.push_back(i);
            continue;
        }
        std::vector<int32_t> vis;
        bool keep = true;
        for (int32_t ch : b.children) {
            const BlockHost &cb = ctx->blocks[(size_t)ch];
            if (!block_in_view(g, cb)) continue;
            vis.push_back(ch);
            const int k = cb.lod - 1;
            const double tau = (k >= 0 && k < n_lod) ? lod_thresh[k] : 0.0;
            if (!(block_range(g, cb) > tau)) keep = false;
        }
        if (keep) sel.push_back(i);
        else
            for (int32_t ch : vis) stack.push_back(ch);
    }
    depth_sort(ctx, *cam, sel);
    *out_n = (int32_t)sel.size();
    if ((int32_t)sel.size() > cap) return fail(COW_ERR_INVALID_ARG, "cow_select_lod: %d blocks exceed cap %d", (int)sel.size(), cap);
    std::copy(sel.begin(), sel.end(), out_ids);
    return COW_OK;
}

cow_status cow_sort_blocks(const cow_ctx *ctx, const cow_camera *cam, const int32_t *ids, int32_t n, int32_t *out) {
    if (!ctx || !cam || (n > 0 && (!ids || !out)) || n < 0) return fail(COW_ERR_INVALID_ARG, "cow_sort_blocks: bad argument");
    std::vector<int32_t> v(ids, ids + n);
    for (int32_t id : v)
        if (id < 0 || id >= (int32_t)ctx->blocks.size()) return fail(COW_ERR_INVALID_ARG, "block id %d out of range", id);
    depth_sort(ctx, *cam, v);
    std::copy(v.begin(), v.end(), out);
    return COW_OK;
}

cow_status cow_render(cow_ctx *ctx, const cow_camera *cams, int32_t n_views, const int32_t *ids,
                      const int32_t *ids_offsets, const float *mlp, float ert_eps, uint32_t flags, float *out_rgb,
                      float *out_aux, int32_t *out_nsamp, void *stream) {
    COW_NVTX("cow_render");
    g_last_error.clear();
    const bool block_mlp = (flags & COW_FLAG_BLOCK_MLPS) != 0;
    if (!ctx || !cams || n_views < 1 || !ids_offsets || (!mlp && !block_mlp) || !out_rgb)
        return fail(COW_ERR_INVALID_ARG, "cow_render: null argument or n_views < 1");
    if (ids_offsets[n_views] > 0 && !ids) return fail(COW_ERR_INVALID_ARG, "cow_render: null ids");
    if (!(ert_eps >= 0.0f && ert_eps < 1.0f)) return fail(COW_ERR_INVALID_ARG, "ert_eps must be in [0, 1)");
    if (flags & ~(COW_FLAG_MLP_BF16 | COW_FLAG_BLOCK_MLPS)) return fail(COW_ERR_INVALID_ARG, "unknown flags");
    if (block_mlp && (flags & COW_FLAG_MLP_BF16))
        return fail(COW_ERR_INVALID_ARG, "COW_FLAG_BLOCK_MLPS runs the MLPs in FP32: drop COW_FLAG_MLP_BF16");
    if (block_mlp && ctx->n_freq < 0) return fail(COW_ERR_INVALID_ARG, "COW_FLAG_BLOCK_MLPS: no block MLPs set");
    if (((uintptr_t)out_rgb & 3u) || ((uintptr_t)out_aux & 15u)) return fail(COW_ERR_INVALID_ARG, "misaligned output");
    DeviceGuard dg(ctx->device);
    cudaStream_t st = (cudaStream_t)stream;
    ViewPlan plan;
    cow_status rc = plan_views(ctx, cams, n_views, ids, ids_offsets, plan);
    if (rc != COW_OK) return rc;
    const int32_t n_ids = ids_offsets[n_views];
    if ((rc = ensure_resident(ctx, ids, n_ids, st)) != COW_OK) return rc;
    // the views' block records, near to far, contiguous per view: each CTA
    // stages its view's records with one bulk copy
    std::vector<cow::BlockRec> vrecs((size_t)std::max(n_ids, 1));
    for (int32_t k = 0; k < n_ids; k++) vrecs[(size_t)k] = ctx->recs[(size_t)ids[k]];
    const size_t vbytes = plan.recs.size() * sizeof(cow::ViewRec);
    const size_t rbytes = vrecs.size() * sizeof(cow::BlockRec);
    // per-block MLP form: the weights of each view record, parallel to the records
    std::vector<const float *> vmlps(block_mlp ? vrecs.size() : 0);
    for (int32_t k = 0; k < n_ids && block_mlp; k++)
        vmlps[(size_t)k] = (const float *)ctx->block_mlps.p + (int64_t)ids[k] * ctx->block_mlp_nparam;
    const size_t mbytes = vmlps.size() * sizeof(const float *);
    COW_CUDA(ctx->views.reserve(vbytes + rbytes + mbytes));
    std::vector<unsigned char> staging(vbytes + rbytes + mbytes);
    std::memcpy(staging.data(), plan.recs.data(), vbytes);
    std::memcpy(staging.data() + vbytes, vrecs.data(), rbytes);
    if (mbytes) std::memcpy(staging.data() + vbytes + rbytes, vmlps.data(), mbytes);
    COW_CUDA(cudaMemcpyAsync(ctx->views.p, staging.data(), vbytes + rbytes + mbytes, cudaMemcpyHostToDevice, st));
    const float *d_mlp = nullptr;
    if (!block_mlp && (rc = resolve_mlp(ctx, mlp, st, &d_mlp)) != COW_OK) return rc;
    float *rgb, *aux;
    int32_t *ns;
    bool h_rgb, h_aux, h_ns;
    if ((rc = resolve_out(out_rgb, (size_t)plan.n_pix * 12, ctx->out_rgb, &rgb, &h_rgb)) != COW_OK) return rc;
    if ((rc = resolve_out(out_aux, (size_t)plan.n_pix * 32, ctx->out_aux, &aux, &h_aux)) != COW_OK) return rc;
    if ((rc = resolve_out(out_nsamp, (size_t)plan.n_pix * 4, ctx->out_nsamp, &ns, &h_ns)) != COW_OK) return rc;
    cow::MarchArgs a;
    std::memset(&a, 0, sizeof(a));
    a.recs = (const cow::BlockRec *)((unsigned char *)ctx->views.p + vbytes);
    a.views = (const cow::ViewRec *)ctx->views.p;
    a.n_views = n_views;
    a.dtype = kernel_dtype(ctx);
    a.mlp = d_mlp;
    a.ert_eps = ert_eps;
    a.flags = flags;
    a.out_rgb = rgb;
    a.out_aux = aux;
    a.out_nsamp = ns;
    a.err = ctx->d_err;
    a.test_flags = ctx->test_flags;
    a.wait_polls = ctx->wait_polls;
    if (block_mlp) {
        a.block_mlps = (const float *const *)((unsigned char *)ctx->views.p + vbytes + rbytes);
        a.n_freq = ctx->n_freq;
    }
    int32_t max_blk = 0;
    for (const auto &r : plan.recs) max_blk = std::max(max_blk, r.ids_count);
    a.smem_recs = max_blk <= 96 ? max_blk : 0;  // views with more records read them from global memory
    bool any_unbounded = false;
    for (int32_t k = 0; k < n_ids; k++) any_unbounded |= ctx->blocks[(size_t)ids[k]].unb != 0;
    if (ctx->schedule == COW_SCHED_THREAD_CONST && n_ids <= cow::kParamRecs) {
        // the records travel in the launch's parameter buffer
        cow::ParamRecs pr;
        std::memset(&pr, 0, sizeof(pr));
        std::copy(vrecs.begin(), vrecs.begin() + n_ids, pr.r);
        COW_CUDA(cow::launch_march_views(a, plan.n_tiles, cow::kSchedThreadConst, st, &pr));
    } else {
        // the warp schedule marches bounded blocks only
        COW_CUDA(cow::launch_march_views(a, plan.n_tiles,
                                         ctx->schedule == COW_SCHED_WARP && !any_unbounded ? cow::kSchedWarp
                                                                                           : cow::kSchedThread, st));
    }
    if ((rc = note_use_impl(ctx, ids, n_ids, st)) != COW_OK) return rc;
    if (h_rgb) COW_CUDA(cudaMemcpyAsync(out_rgb, rgb, (size_t)plan.n_pix * 12, cudaMemcpyDeviceToHost, st));
    if (h_aux) COW_CUDA(cudaMemcpyAsync(out_aux, aux, (size_t)plan.n_pix * 32, cudaMemcpyDeviceToHost, st));
    if (h_ns) COW_CUDA(cudaMemcpyAsync(out_nsamp, ns, (size_t)plan.n_pix * 4, cudaMemcpyDeviceToHost, st));
    return COW_OK;
}

static cow_status render_rays_impl(cow_ctx *ctx, const float *o, const float *d, int64_t n_rays, const int32_t *ids,
                                   int32_t n_ids, const float *mlp, float ert_eps, uint32_t flags, float *out_rgb,
                                   float *out_aux, int32_t *out_nsamp, float *out_block_T, void *stream,
                                   float *out_block_state = nullptr) {
    COW_NVTX("cow_render_rays");
    g_last_error.clear();
    if (ctx && n_rays == 0) return COW_OK;  // an empty batch (its arrays may be NULL)
    const bool block_mlp = (flags & COW_FLAG_BLOCK_MLPS) != 0;
    if (!ctx || !o || !d || n_rays < 0 || !ids || (!mlp && !block_mlp) || !out_rgb)
        return fail(COW_ERR_INVALID_ARG, "cow_render_rays: null argument");
    if (n_ids < 1 || n_ids > cow::kMaxRayIds) return fail(COW_ERR_INVALID_ARG, "n_ids must be in [1, %d]", cow::kMaxRayIds);
    if (!(ert_eps >= 0.0f && ert_eps < 1.0f)) return fail(COW_ERR_INVALID_ARG, "ert_eps must be in [0, 1)");
    if (flags & ~(COW_FLAG_MLP_BF16 | COW_FLAG_BLOCK_MLPS)) return fail(COW_ERR_INVALID_ARG, "unknown flags");
    if (block_mlp && (flags & COW_FLAG_MLP_BF16))
        return fail(COW_ERR_INVALID_ARG, "COW_FLAG_BLOCK_MLPS runs the MLPs in FP32: drop COW_FLAG_MLP_BF16");
    if (block_mlp && ctx->n_freq < 0)
        return fail(COW_ERR_INVALID_ARG, "COW_FLAG_BLOCK_MLPS: no per-block MLPs set (cow_set_block_mlps)");
    if (block_mlp && out_block_T)
        return fail(COW_ERR_INVALID_ARG, "in-block transmittances are kept for the global-MLP form only");
    for (int32_t k = 0; k < n_ids; k++)
        if (ids[k] < 0 || ids[k] >= (int32_t)ctx->blocks.size()) return fail(COW_ERR_INVALID_ARG, "block id %d out of range", ids[k]);
    if (!is_device_ptr(o) || !is_device_ptr(d)) return fail(COW_ERR_INVALID_ARG, "ray origins and directions must be device memory");
    if (((uintptr_t)out_rgb & 3u) || ((uintptr_t)out_aux & 15u)) return fail(COW_ERR_INVALID_ARG, "misaligned output");
    DeviceGuard dg(ctx->device);
    cudaStream_t st = (cudaStream_t)stream;
    cow_status rc;
    if ((rc = ensure_resident(ctx, ids, n_ids, st)) != COW_OK) return rc;
    const float *d_mlp = nullptr;
    if (!block_mlp && (rc = resolve_mlp(ctx, mlp, st, &d_mlp)) != COW_OK) return rc;
    float *rgb, *aux;
    int32_t *ns;
    bool h_rgb, h_aux, h_ns;
    if ((rc = resolve_out(out_rgb, (size_t)n_rays * 12, ctx->out_rgb, &rgb, &h_rgb)) != COW_OK) return rc;
    if ((rc = resolve_out(out_aux, (size_t)n_rays * 32, ctx->out_aux, &aux, &h_aux)) != COW_OK) return rc;
    if ((rc = resolve_out(out_nsamp, (size_t)n_rays * 4, ctx->out_nsamp, &ns, &h_ns)) != COW_OK) return rc;
    cow::MarchArgs a;
    std::memset(&a, 0, sizeof(a));
    a.dtype = kernel_dtype(ctx);
    a.mlp = d_mlp;
    a.ert_eps = ert_eps;
    a.flags = flags;
    a.out_rgb = rgb;
    a.out_aux = aux;
    a.out_nsamp = ns;
    a.err = ctx->d_err;
    a.test_flags = ctx->test_flags;
    a.wait_polls = ctx->wait_polls;
    a.ray_o = o;
    a.ray_d = d;
    a.n_rays = n_rays;
    a.out_block_T = out_block_T;
    a.out_block_state = out_block_state;
    if (block_mlp) {
        a.block_mlp_base = (const float *)ctx->block_mlps.p;
        a.block_mlp_stride = ctx->block_mlp_nparam;
        a.n_freq = ctx->n_freq;
    }
    if ((rc = ray_order(ctx, o, d, n_rays, ids, n_ids, st, &a.ray_perm)) != COW_OK) return rc;
    cow::RayRecs rr;
    make_ray_recs(ctx, ids, n_ids, rr);
    COW_CUDA(cow::launch_march_rays(a, rr, st));
    if ((rc = note_use_impl(ctx, ids, n_ids, st)) != COW_OK) return rc;
    if (h_rgb) COW_CUDA(cudaMemcpyAsync(out_rgb, rgb, (size_t)n_rays * 12, cudaMemcpyDeviceToHost, st));
    if (h_aux) COW_CUDA(cudaMemcpyAsync(out_aux, aux, (size_t)n_rays * 32, cudaMemcpyDeviceToHost, st));
    if (h_ns) COW_CUDA(cudaMemcpyAsync(out_nsamp, ns, (size_t)n_rays * 4, cudaMemcpyDeviceToHost, st));
    return COW_OK;
}

cow_status cow_render_partials(cow_ctx *ctx, const float *o, const float *d, int64_t n_rays, const int32_t *ids,
                               int32_t n_ids, float *out_partials, void *stream) {
    COW_NVTX("cow_render_partials");
    g_last_error.clear();
    if (ctx && n_rays == 0) return COW_OK;  // an empty batch (its arrays may be NULL)
    if (!ctx || !o || !d || n_rays < 0 || !ids || !out_partials)
        return fail(COW_ERR_INVALID_ARG, "cow_render_partials: null argument");
    if (n_ids < 1 || n_ids > cow::kMaxRayIds) return fail(COW_ERR_INVALID_ARG, "n_ids must be in [1, %d]", cow::kMaxRayIds);
    for (int32_t k = 0; k < n_ids; k++)
        if (ids[k] < 0 || ids[k] >= (int32_t)ctx->blocks.size()) return fail(COW_ERR_INVALID_ARG, "block id %d out of range", ids[k]);
    for (const void *q : {(const void *)o, (const void *)d, (const void *)out_partials})
        if (!is_device_ptr(q)) return fail(COW_ERR_INVALID_ARG, "rays and partials must be device memory");
    if ((uintptr_t)out_partials & 15u) return fail(COW_ERR_INVALID_ARG, "partials must be 16-byte aligned");
    DeviceGuard dg(ctx->device);
    cudaStream_t st = (cudaStream_t)stream;
    cow_status rc;
    if ((rc = ensure_resident(ctx, ids, n_ids, st)) != COW_OK) return rc;
    cow::MarchArgs a;
    std::memset(&a, 0, sizeof(a));
    a.dtype = kernel_dtype(ctx);
    a.err = ctx->d_err;
    a.ray_o = o;
    a.ray_d = d;
    a.n_rays = n_rays;
    a.out_partials = out_partials;
    if ((rc = ray_order(ctx, o, d, n_rays, ids, n_ids, st, &a.ray_perm)) != COW_OK) return rc;
    cow::RayRecs rr;
    make_ray_recs(ctx, ids, n_ids, rr);
    COW_CUDA(cow::launch_march_partials(a, rr, st));
    return note_use_impl(ctx, ids, n_ids, st);
}

cow_status cow_composite_over(cow_ctx *ctx, const float *o, const float *d, int64_t n_rays, const int32_t *ids,
                              int32_t n_ids, const float *partials, const float *mlp, uint32_t flags, float *out_rgb,
                              float *out_aux, void *stream) {
    COW_NVTX("cow_composite_over");
    g_last_error.clear();
    if (ctx && n_rays == 0) return COW_OK;  // an empty batch (its arrays may be NULL)
    if (!ctx || !o || !d || n_rays < 0 || !ids || !partials || !mlp || !out_rgb)
        return fail(COW_ERR_INVALID_ARG, "cow_composite_over: null argument");
    if (n_ids < 1 || n_ids > cow::kMaxRayIds) return fail(COW_ERR_INVALID_ARG, "n_ids must be in [1, %d]", cow::kMaxRayIds);
    if (flags & ~COW_FLAG_MLP_BF16) return fail(COW_ERR_INVALID_ARG, "unknown flags");
    for (int32_t k = 0; k < n_ids; k++)
        if (ids[k] < 0 || ids[k] >= (int32_t)ctx->blocks.size()) return fail(COW_ERR_INVALID_ARG, "block id %d out of range", ids[k]);
    for (const void *q : {(const void *)o, (const void *)d, (const void *)partials, (const void *)out_rgb})
        if (!is_device_ptr(q)) return fail(COW_ERR_INVALID_ARG, "rays, partials and outputs must be device memory");
    if (out_aux && (!is_device_ptr(out_aux) || ((uintptr_t)out_aux & 15u)))
        return fail(COW_ERR_INVALID_ARG, "aux must be 16-byte aligned device memory");
    if (((uintptr_t)partials & 15u) || ((uintptr_t)out_rgb & 3u)) return fail(COW_ERR_INVALID_ARG, "misaligned array");
    DeviceGuard dg(ctx->device);
    cudaStream_t st = (cudaStream_t)stream;
    const float *d_mlp = nullptr;
    cow_status rc;
    if ((rc = resolve_mlp(ctx, mlp, st, &d_mlp)) != COW_OK) return rc;
    cow::MarchArgs a;
    std::memset(&a, 0, sizeof(a));
    a.mlp = d_mlp;
    a.flags = flags;
    a.out_rgb = out_rgb;
    a.out_aux = out_aux;
    a.err = ctx->d_err;
    a.ray_o = o;
    a.ray_d = d;
    a.n_rays = n_rays;
    a.in_partials = partials;
    cow::RayRecs rr;
    make_ray_recs(ctx, ids, n_ids, rr);  // only the blocks' centres are read (the per-ray order)
    COW_CUDA(cow::launch_composite_over(a, rr, st));
    return COW_OK;
}

cow_status cow_render_rays_f64(cow_ctx *ctx, const float *o, const float *d, int64_t n_rays, const int32_t *ids,
                               int32_t n_ids, const double *mlp, const double *const *grids,
                               const double *const *planes, double *out_rgb, double *out_aux, void *stream) {
    g_last_error.clear();
    if (ctx && n_rays == 0) return COW_OK;
    if (!ctx || !o || !d || n_rays < 0 || !ids || !mlp || !grids || !planes || !out_rgb)
        return fail(COW_ERR_INVALID_ARG, "cow_render_rays_f64: null argument");
    if (n_ids < 1 || n_ids > cow::kMaxRayIds) return fail(COW_ERR_INVALID_ARG, "n_ids must be in [1, %d]", cow::kMaxRayIds);
    const int32_t nb = (int32_t)ctx->blocks.size();
    for (int32_t k = 0; k < n_ids; k++) {
        if (ids[k] < 0 || ids[k] >= nb) return fail(COW_ERR_INVALID_ARG, "block id %d out of range", ids[k]);
        const int32_t id = ids[k];
        for (int q = 0; q < 4; q++) {
            const void *p = q == 0 ? (const void *)grids[id] : (const void *)planes[3 * id + q - 1];
            if (!p || !is_device_ptr(p)) return fail(COW_ERR_INVALID_ARG, "block %d: FP64 features must be device memory", id);
        }
    }
    for (const void *q : {(const void *)o, (const void *)d, (const void *)mlp, (const void *)out_rgb})
        if (!is_device_ptr(q)) return fail(COW_ERR_INVALID_ARG, "rays, MLP and outputs must be device memory");
    if (out_aux && !is_device_ptr(out_aux)) return fail(COW_ERR_INVALID_ARG, "aux must be device memory");
    DeviceGuard dg(ctx->device);
    cudaStream_t st = (cudaStream_t)stream;
    cow_status rc;
    if ((rc = ensure_resident(ctx, ids, n_ids, st)) != COW_OK) return rc;  // the records' occupancy and tables
    std::vector<const double *> tab((size_t)nb * 4, nullptr);
    for (int32_t i = 0; i < nb; i++) {
        tab[(size_t)i] = grids[i];
        for (int q = 0; q < 3; q++) tab[(size_t)nb + 3 * (size_t)i + q] = planes[3 * i + q];
    }
    COW_CUDA(ctx->f64ptrs.reserve(tab.size() * sizeof(double *)));
    COW_CUDA(cudaMemcpyAsync(ctx->f64ptrs.p, tab.data(), tab.size() * sizeof(double *), cudaMemcpyHostToDevice, st));
    cow::F64Args a;
    std::memset(&a, 0, sizeof(a));
    a.ray_o = o;
    a.ray_d = d;
    a.n_rays = n_rays;
    a.grids = (const double *const *)ctx->f64ptrs.p;
    a.planes = (const double *const *)ctx->f64ptrs.p + nb;
    a.mlp = mlp;
    a.out_rgb = out_rgb;
    a.out_aux = out_aux;
    a.err = ctx->d_err;
    cow::RayRecs rr;
    make_ray_recs(ctx, ids, n_ids, rr);
    COW_CUDA(cow::launch_march_rays_f64(a, rr, st));
    COW_CUDA(cudaStreamSynchronize(st));  // the host pointer table is reused by the next call
    return note_use_impl(ctx, ids, n_ids, st);
}

cow_status cow_render_rays(cow_ctx *ctx, const float *o, const float *d, int64_t n_rays, const int32_t *ids,
                           int32_t n_ids, const float *mlp, float ert_eps, uint32_t flags, float *out_rgb,
                           float *out_aux, int32_t *out_nsamp, void *stream) {
    return render_rays_impl(ctx, o, d, n_rays, ids, n_ids, mlp, ert_eps, flags, out_rgb, out_aux, out_nsamp, nullptr,
                            stream);
}

cow_status cow_render_rays_block_t(cow_ctx *ctx, const float *o, const float *d, int64_t n_rays, const int32_t *ids,
                                   int32_t n_ids, const float *mlp, uint32_t flags, float *out_rgb, float *out_aux,
                                   int32_t *out_nsamp, float *out_block_T, void *stream) {
    g_last_error.clear();
    if (ctx && n_rays == 0) return COW_OK;
    if (!out_block_T || !is_device_ptr(out_block_T))
        return fail(COW_ERR_INVALID_ARG, "out_block_T must be device memory (n_rays x n_ids floats)");
    return render_rays_impl(ctx, o, d, n_rays, ids, n_ids, mlp, 0.0f, flags, out_rgb, out_aux, out_nsamp, out_block_T,
                            stream);
}

cow_status cow_render_rays_block_state(cow_ctx *ctx, const float *o, const float *d, int64_t n_rays,
                                       const int32_t *ids, int32_t n_ids, float *out_rgb, float *out_state,
                                       void *stream) {
    g_last_error.clear();
    if (ctx && n_rays == 0) return COW_OK;
    if (!out_state || !is_device_ptr(out_state) || ((uintptr_t)out_state & 15u))
        return fail(COW_ERR_INVALID_ARG, "out_state must be 16-byte aligned device memory (n_rays x n_ids x 8 floats)");
    return render_rays_impl(ctx, o, d, n_rays, ids, n_ids, nullptr, 0.0f, COW_FLAG_BLOCK_MLPS, out_rgb, nullptr,
                            nullptr, nullptr, stream, out_state);
}

cow_status cow_render_backward(cow_ctx *ctx, const float *o, const float *d, int64_t n_rays, const int32_t *ids,
                               int32_t n_ids, const float *mlp, float ert_eps, const float *aux, const float *dL_drgb,
                               float *const *grad_grid, float *const *grad_planes, float *grad_mlp, void *stream) {
    COW_NVTX("cow_render_backward");
    g_last_error.clear();
    if (ctx && n_rays == 0) return COW_OK;  // an empty batch (its arrays may be NULL)
    if (!ctx || !o || !d || n_rays < 0 || !ids || !mlp || !aux || !dL_drgb || !grad_grid || !grad_planes || !grad_mlp)
        return fail(COW_ERR_INVALID_ARG, "cow_render_backward: null argument");
    if (n_ids < 1 || n_ids > cow::kMaxRayIds) return fail(COW_ERR_INVALID_ARG, "n_ids must be in [1, %d]", cow::kMaxRayIds);
    if (!(ert_eps >= 0.0f && ert_eps < 1.0f)) return fail(COW_ERR_INVALID_ARG, "ert_eps must be in [0, 1)");
    const int32_t nb = (int32_t)ctx->blocks.size();
    for (int32_t k = 0; k < n_ids; k++)
        if (ids[k] < 0 || ids[k] >= nb) return fail(COW_ERR_INVALID_ARG, "block id %d out of range", ids[k]);
    for (const void *q : {(const void *)o, (const void *)d, (const void *)aux, (const void *)dL_drgb, (const void *)grad_mlp, (const void *)mlp})
        if (!is_device_ptr(q)) return fail(COW_ERR_INVALID_ARG, "backward arrays and the MLP must be device memory");
    if (((uintptr_t)aux & 15u)) return fail(COW_ERR_INVALID_ARG, "aux must be 16-byte aligned");
    std::vector<float *> ptrs((size_t)nb * 4);
    for (int32_t i = 0; i < nb; i++) {
        ptrs[(size_t)i] = grad_grid[i];
        for (int k = 0; k < 3; k++) ptrs[(size_t)nb + 3 * (size_t)i + k] = grad_planes[3 * i + k];
        for (int k = 0; k < 4; k++) {
            const float *q = k == 0 ? grad_grid[i] : grad_planes[3 * i + k - 1];
            if (q && (((uintptr_t)q & 15u) || !is_device_ptr(q)))
                return fail(COW_ERR_INVALID_ARG, "block %d: gradient arrays must be 16-byte aligned device memory", i);
        }
    }
    DeviceGuard dg(ctx->device);
    cudaStream_t st = (cudaStream_t)stream;
    cow_status rc = ensure_resident(ctx, ids, n_ids, st);
    if (rc != COW_OK) return rc;
    COW_CUDA(ctx->gptrs.reserve(ptrs.size() * sizeof(float *)));
    COW_CUDA(cudaMemcpyAsync(ctx->gptrs.p, ptrs.data(), ptrs.size() * sizeof(float *), cudaMemcpyHostToDevice, st));
    const int rows = cow::backward_rows(n_rays);
    const size_t part_bytes = ((size_t)std::max(rows, 1) * cow::kMlpParams * sizeof(float) + 255) & ~(size_t)255;
    COW_CUDA(ctx->partials.reserve(part_bytes + (size_t)std::max<int64_t>(n_rays, 1) * 8 * sizeof(float)));
    cow::BwdArgs a;
    std::memset(&a, 0, sizeof(a));
    a.dtype = kernel_dtype(ctx);
    a.mlp = mlp;
    a.ert_eps = ert_eps;
    a.ray_o = o;
    a.ray_d = d;
    a.n_rays = n_rays;
    a.aux = aux;
    a.dL_drgb = dL_drgb;
    a.grad_grid = (float *const *)ctx->gptrs.p;
    a.grad_planes = (float *const *)ctx->gptrs.p + nb;
    a.grad_mlp = grad_mlp;
    a.partials = (float *)ctx->partials.p;
    a.gcf = (float *)((unsigned char *)ctx->partials.p + part_bytes);
    a.err = ctx->d_err;
    if ((rc = ray_order(ctx, o, d, n_rays, ids, n_ids, st, &a.ray_perm)) != COW_OK) return rc;
    cow::RayRecs rr;
    make_ray_recs(ctx, ids, n_ids, rr);
    COW_CUDA(cow::launch_backward_rays(a, rr, st));
    return note_use_impl(ctx, ids, n_ids, st);
}

static cow_status backward_block_mlps_impl(cow_ctx *ctx, const float *o, const float *d, int64_t n_rays,
                                           const int32_t *ids, int32_t n_ids, const float *state,
                                           const float *dL_drgb, float *const *grad_grid, float *const *grad_planes,
                                           float *grad_block_mlps, void *stream) {
    COW_NVTX("cow_render_backward_block_mlps");
    g_last_error.clear();
    if (state && (!is_device_ptr(state) || ((uintptr_t)state & 15u)))
        return fail(COW_ERR_INVALID_ARG, "state must be 16-byte aligned device memory (n_rays x n_ids x 8 floats)");
    if (ctx && n_rays == 0) return COW_OK;  // an empty batch (its arrays may be NULL)
    if (!ctx || !o || !d || n_rays < 0 || !ids || !dL_drgb || !grad_grid || !grad_planes || !grad_block_mlps)
        return fail(COW_ERR_INVALID_ARG, "cow_render_backward_block_mlps: null argument");
    if (ctx->n_freq < 0) return fail(COW_ERR_INVALID_ARG, "no per-block MLPs set (cow_set_block_mlps)");
    if (n_ids < 1 || n_ids > cow::kMaxRayIds) return fail(COW_ERR_INVALID_ARG, "n_ids must be in [1, %d]", cow::kMaxRayIds);
    const int32_t nb = (int32_t)ctx->blocks.size();
    for (int32_t k = 0; k < n_ids; k++)
        if (ids[k] < 0 || ids[k] >= nb) return fail(COW_ERR_INVALID_ARG, "block id %d out of range", ids[k]);
    for (const void *q : {(const void *)o, (const void *)d, (const void *)dL_drgb, (const void *)grad_block_mlps})
        if (!is_device_ptr(q)) return fail(COW_ERR_INVALID_ARG, "backward arrays must be device memory");
    if ((uintptr_t)grad_block_mlps & 3u) return fail(COW_ERR_INVALID_ARG, "grad_block_mlps must be 4-byte aligned");
    if (n_rays > ((int64_t)1 << 40) / ((int64_t)n_ids * 64))
        return fail(COW_ERR_INVALID_ARG, "too many rays x blocks for one call");
    std::vector<float *> ptrs((size_t)nb * 4);
    for (int32_t i = 0; i < nb; i++) {
        ptrs[(size_t)i] = grad_grid[i];
        for (int k = 0; k < 3; k++) ptrs[(size_t)nb + 3 * (size_t)i + k] = grad_planes[3 * i + k];
        for (int k = 0; k < 4; k++) {
            const float *q = k == 0 ? grad_grid[i] : grad_planes[3 * i + k - 1];
            if (q && (((uintptr_t)q & 15u) || !is_device_ptr(q)))
                return fail(COW_ERR_INVALID_ARG, "block %d: gradient arrays must be 16-byte aligned device memory", i);
        }
    }
    DeviceGuard dg(ctx->device);
    cudaStream_t st = (cudaStream_t)stream;
    cow_status rc = ensure_resident(ctx, ids, n_ids, st);
    if (rc != COW_OK) return rc;
    COW_CUDA(ctx->gptrs.reserve(ptrs.size() * sizeof(float *)));
    COW_CUDA(cudaMemcpyAsync(ctx->gptrs.p, ptrs.data(), ptrs.size() * sizeof(float *), cudaMemcpyHostToDevice, st));
    const size_t half = (size_t)n_rays * (size_t)n_ids * 8 * sizeof(float);
    COW_CUDA(ctx->bm_scratch.reserve(state ? half : 2 * half));
    const int32_t n_in = 10 + 6 * ctx->n_freq;
    cow::BmBwdArgs a;
    std::memset(&a, 0, sizeof(a));
    a.dtype = kernel_dtype(ctx);
    a.ray_o = o;
    a.ray_d = d;
    a.n_rays = n_rays;
    a.dL_drgb = dL_drgb;
    a.grad_grid = (float *const *)ctx->gptrs.p;
    a.grad_planes = (float *const *)ctx->gptrs.p + nb;
    a.mlps = (const float *)ctx->block_mlps.p;
    a.mlp_stride = ctx->block_mlp_nparam;
    a.grad_mlps = grad_block_mlps;
    a.grad_stride = 16 * n_in + 16 + 16 * 16 + 16 + 16 * 3 + 3;
    a.n_freq = ctx->n_freq;
    a.n_ids = n_ids;
    // S: the forward's per-block state when given (the first pass is then
    // skipped), else scratch; G: scratch
    a.S = state ? const_cast<float *>(state) : (float *)ctx->bm_scratch.p;
    a.G = state ? (float *)ctx->bm_scratch.p : (float *)((unsigned char *)ctx->bm_scratch.p + half);
    a.have_state = state ? 1 : 0;
    a.err = ctx->d_err;
    if ((rc = ray_order(ctx, o, d, n_rays, ids, n_ids, st, &a.ray_perm)) != COW_OK) return rc;
    cow::RayRecs rr;
    make_ray_recs(ctx, ids, n_ids, rr);
    COW_CUDA(cow::launch_backward_block_mlps(a, rr, st));
    return note_use_impl(ctx, ids, n_ids, st);
}

cow_status cow_render_backward_block_mlps(cow_ctx *ctx, const float *o, const float *d, int64_t n_rays,
                                          const int32_t *ids, int32_t n_ids, const float *dL_drgb,
                                          float *const *grad_grid, float *const *grad_planes, float *grad_block_mlps,
                                          void *stream) {
    return backward_block_mlps_impl(ctx, o, d, n_rays, ids, n_ids, nullptr, dL_drgb, grad_grid, grad_planes,
                                    grad_block_mlps, stream);
}

cow_status cow_render_backward_block_mlps_state(cow_ctx *ctx, const float *o, const float *d, int64_t n_rays,
                                                const int32_t *ids, int32_t n_ids, const float *state,
                                                const float *dL_drgb, float *const *grad_grid,
                                                float *const *grad_planes, float *grad_block_mlps, void *stream) {
    g_last_error.clear();
    if (ctx && n_rays > 0 && !state) return fail(COW_ERR_INVALID_ARG, "null state");
    return backward_block_mlps_impl(ctx, o, d, n_rays, ids, n_ids, state, dL_drgb, grad_grid, grad_planes,
                                    grad_block_mlps, stream);
}

namespace {

// Validate the ids and the per-block gradient arrays of a regulariser call,
// load the blocks and upload the gradient pointer table.
cow_status reg_prepare(cow_ctx *ctx, const int32_t *ids, int32_t n_ids, float *loss, float *const *grad_grid,
                       float *const *grad_planes, cudaStream_t st, cow::RegArgs &a) {
    if (n_ids < 1 || n_ids > cow::kMaxRayIds) return fail(COW_ERR_INVALID_ARG, "n_ids must be in [1, %d]", cow::kMaxRayIds);
    const int32_t nb = (int32_t)ctx->blocks.size();
    for (int32_t k = 0; k < n_ids; k++)
        if (ids[k] < 0 || ids[k] >= nb) return fail(COW_ERR_INVALID_ARG, "block id %d out of range", ids[k]);
    if (loss && !is_device_ptr(loss)) return fail(COW_ERR_INVALID_ARG, "loss must be device memory");
    if ((grad_grid == nullptr) != (grad_planes == nullptr))
        return fail(COW_ERR_INVALID_ARG, "pass both gradient tables or neither");
    std::memset(&a, 0, sizeof(a));
    cow_status rc = ensure_resident(ctx, ids, n_ids, st);
    if (rc != COW_OK) return rc;
    if (grad_grid) {
        std::vector<float *> ptrs((size_t)nb * 4);
        for (int32_t i = 0; i < nb; i++) {
            ptrs[(size_t)i] = grad_grid[i];
            for (int k = 0; k < 3; k++) ptrs[(size_t)nb + 3 * (size_t)i + k] = grad_planes[3 * i + k];
            for (int k = 0; k < 4; k++) {
                const float *q = k == 0 ? grad_grid[i] : grad_planes[3 * i + k - 1];
                if (q && (((uintptr_t)q & 3u) || !is_device_ptr(q)))
                    return fail(COW_ERR_INVALID_ARG, "block %d: gradient arrays must be aligned device memory", i);
            }
        }
        COW_CUDA(ctx->gptrs.reserve(ptrs.size() * sizeof(float *)));
        COW_CUDA(cudaMemcpyAsync(ctx->gptrs.p, ptrs.data(), ptrs.size() * sizeof(float *), cudaMemcpyHostToDevice, st));
        a.grad_grid = (float *const *)ctx->gptrs.p;
        a.grad_planes = (float *const *)ctx->gptrs.p + nb;
    }
    a.dtype = kernel_dtype(ctx);
    a.loss = loss;
    a.err = ctx->d_err;
    return COW_OK;
}

}  // namespace

cow_status cow_sparsity_loss(cow_ctx *ctx, const float *points, int64_t n_points, const int32_t *ids, int32_t n_ids,
                             float weight, float *loss, float *const *grad_grid, float *const *grad_planes,
                             void *stream) {
    COW_NVTX("cow_sparsity_loss");
    g_last_error.clear();
    if (ctx && n_points == 0) return COW_OK;  // nothing to add (the arrays may be NULL)
    if (!ctx || !points || n_points < 0 || !ids) return fail(COW_ERR_INVALID_ARG, "cow_sparsity_loss: null argument");
    if (!is_device_ptr(points)) return fail(COW_ERR_INVALID_ARG, "points must be device memory");
    if (ctx->bricks)
        return fail(COW_ERR_UNSUPPORTED, "the sparsity regulariser samples arbitrary points, and a brick-sparse grid "
                    "keeps only the bricks with occupied cells");
    DeviceGuard dg(ctx->device);
    cudaStream_t st = (cudaStream_t)stream;
    cow::RegArgs a;
    cow_status rc = reg_prepare(ctx, ids, n_ids, loss, grad_grid, grad_planes, st, a);
    if (rc != COW_OK) return rc;
    a.pts = points;
    a.n = n_points;
    a.weight = weight;
    cow::RayRecs rr;
    make_ray_recs(ctx, ids, n_ids, rr);
    COW_CUDA(cow::launch_sparsity(a, rr, st));
    return note_use_impl(ctx, ids, n_ids, st);
}

cow_status cow_opacity_loss(cow_ctx *ctx, const float *o, const float *d, int64_t n_rays, const int32_t *ids,
                            int32_t n_ids, const float *block_T, float weight, float *loss, float *const *grad_grid,
                            float *const *grad_planes, void *stream) {
    COW_NVTX("cow_opacity_loss");
    g_last_error.clear();
    if (ctx && n_rays == 0) return COW_OK;  // nothing to add (the arrays may be NULL)
    if (!ctx || !o || !d || n_rays < 0 || !ids) return fail(COW_ERR_INVALID_ARG, "cow_opacity_loss: null argument");
    if (!is_device_ptr(o) || !is_device_ptr(d)) return fail(COW_ERR_INVALID_ARG, "rays must be device memory");
    DeviceGuard dg(ctx->device);
    cudaStream_t st = (cudaStream_t)stream;
    cow::RegArgs a;
    cow_status rc = reg_prepare(ctx, ids, n_ids, loss, grad_grid, grad_planes, st, a);
    if (rc != COW_OK) return rc;
    if (block_T && !is_device_ptr(block_T)) return fail(COW_ERR_INVALID_ARG, "block_T must be device memory");
    a.ray_o = o;
    a.ray_d = d;
    a.n = n_rays;
    a.weight = weight;
    a.block_T = block_T;
    if ((rc = ray_order(ctx, o, d, n_rays, ids, n_ids, st, &a.ray_perm)) != COW_OK) return rc;
    cow::RayRecs rr;
    make_ray_recs(ctx, ids, n_ids, rr);
    COW_CUDA(cow::launch_opacity(a, rr, st));
    return note_use_impl(ctx, ids, n_ids, st);
}

cow_status cow_update_features(cow_ctx *ctx, int32_t block, const float *grid, const float *plane_xy,
                               const float *plane_xz, const float *plane_yz, void *stream) {
    COW_NVTX("cow_update_features");
    g_last_error.clear();
    if (!ctx || !grid || !plane_xy || !plane_xz || !plane_yz) return fail(COW_ERR_INVALID_ARG, "null argument");
    if (block < 0 || block >= (int32_t)ctx->blocks.size()) return fail(COW_ERR_INVALID_ARG, "block out of range");
    for (const float *q : {grid, plane_xy, plane_xz, plane_yz})
        if (((uintptr_t)q & 15u) != 0) return fail(COW_ERR_INVALID_ARG, "arrays must be 16-byte aligned");
    DeviceGuard dg(ctx->device);
    cudaStream_t st = (cudaStream_t)stream;
    BlockHost &b = ctx->blocks[(size_t)block];
    const size_t need = (size_t)std::max((int64_t)b.R * b.R * b.R, (int64_t)b.P * b.P) * 32;
    // staging (host masters) and small scratch for the FP8 scale search
    COW_CUDA(ctx->staging.reserve(need + 256));
    unsigned *d_amax = (unsigned *)((unsigned char *)ctx->staging.p + need);
    float *d_inv = (float *)((unsigned char *)ctx->staging.p + need + 64);
    const float *src[4] = {grid, plane_xy, plane_xz, plane_yz};
    cow_status rc = ensure_resident(ctx, &block, 1, st);
    if (rc != COW_OK) return rc;
    rc = repack_block(ctx, b, src, ctx->staging.p, d_amax, d_inv, st);
    if (rc == COW_OK && ctx->budget > 0) {
        b.dirty = true;
        rc = note_use_impl(ctx, &block, 1, st);  // an unload waits for the re-pack (and writes it back)
    }
    return rc;
}

cow_status cow_adam_step(float *param, const float *grad, float *m, float *v, int64_t n, float lr, float beta1,
                         float beta2, float eps, int32_t step, void *stream) {
    if (!param || !grad || !m || !v || n < 0 || step < 1 || !(lr >= 0.f) || !(beta1 >= 0.f && beta1 < 1.f) ||
        !(beta2 >= 0.f && beta2 < 1.f) || !(eps > 0.f))
        return fail(COW_ERR_INVALID_ARG, "cow_adam_step: bad argument");
    COW_CUDA(cow::launch_adam(param, grad, m, v, n, lr, beta1, beta2, eps, step, (cudaStream_t)stream));
    return COW_OK;
}

cow_status cow_mse_grad(const float *rgb, const float *target, int64_t n, float *dL_drgb, float *loss, void *stream) {
    if (!rgb || !target || !dL_drgb || n < 0) return fail(COW_ERR_INVALID_ARG, "cow_mse_grad: bad argument");
    COW_CUDA(cow::launch_mse_grad(rgb, target, n, dL_drgb, loss, (cudaStream_t)stream));
    return COW_OK;
}

cow_status cow_set_block_mlps(cow_ctx *ctx, const float *mlps, int32_t n_mlps, int32_t n_freq, void *stream) {
    g_last_error.clear();
    if (!ctx) return fail(COW_ERR_INVALID_ARG, "null context");
    if (!mlps && n_mlps == 0) {
        ctx->n_freq = -1;
        ctx->block_mlp_nparam = 0;
        return COW_OK;
    }
    if (!mlps) return fail(COW_ERR_INVALID_ARG, "cow_set_block_mlps: null mlps");
    if (n_mlps != (int32_t)ctx->blocks.size())
        return fail(COW_ERR_INVALID_ARG, "cow_set_block_mlps: %d MLPs for %d blocks", n_mlps, (int)ctx->blocks.size());
    if (n_freq < 0 || n_freq > 8) return fail(COW_ERR_INVALID_ARG, "n_freq must be in [0, 8]");
    DeviceGuard dg(ctx->device);
    cudaStream_t st = (cudaStream_t)stream;
    const int32_t n_in = 10 + 6 * n_freq;
    const int32_t np = 16 * n_in + 16 + 16 * 16 + 16 + 16 * 3 + 3;
    // the kernel reads W1 / W2 rows as float4: each block's copy starts on a
    // 16-byte boundary (stride rounded up to 4 floats)
    const int32_t stride = (np + 3) & ~3;
    COW_CUDA(ctx->block_mlps.reserve((size_t)n_mlps * (size_t)stride * sizeof(float)));
    COW_CUDA(cudaMemcpy2DAsync(ctx->block_mlps.p, (size_t)stride * sizeof(float), mlps, (size_t)np * sizeof(float),
                               (size_t)np * sizeof(float), (size_t)n_mlps,
                               is_device_ptr(mlps) ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice, st));
    ctx->n_freq = n_freq;
    ctx->block_mlp_nparam = stride;
    return COW_OK;
}

cow_status cow_set_block_unbounded(cow_ctx *ctx, int32_t block, int32_t flags, void *stream) {
    g_last_error.clear();
    if (!ctx) return fail(COW_ERR_INVALID_ARG, "null context");
    if (block < 0 || block >= (int32_t)ctx->blocks.size()) return fail(COW_ERR_INVALID_ARG, "block out of range");
    if (flags & ~31) return fail(COW_ERR_INVALID_ARG, "unknown unbounded flags %d", flags);
    if (flags && !(flags & COW_UNBOUNDED_CONTRACTED))
        return fail(COW_ERR_INVALID_ARG, "extended sides need COW_UNBOUNDED_CONTRACTED");
    DeviceGuard dg(ctx->device);
    cudaStream_t st = (cudaStream_t)stream;
    COW_CUDA(cudaStreamSynchronize(st));  // earlier calls may still read the record
    ctx->blocks[(size_t)block].unb = flags;
    return refresh_rec(ctx, block, st);
}

cow_status cow_set_residency(cow_ctx *ctx, int64_t budget_bytes, void *stream) {
    COW_NVTX("cow_set_residency");
    g_last_error.clear();
    if (!ctx || budget_bytes < 0) return fail(COW_ERR_INVALID_ARG, "cow_set_residency: null context or budget < 0");
    DeviceGuard dg(ctx->device);
    cudaStream_t st = (cudaStream_t)stream;
    COW_CUDA(cudaStreamSynchronize(st));
    if (ctx->copy_stream) COW_CUDA(cudaStreamSynchronize(ctx->copy_stream));
    const int32_t nb = (int32_t)ctx->blocks.size();
    cow_status rc;
    if (budget_bytes > 0) {
        if (!ctx->pool) {
            // the context's own stream-ordered pool: memory of unloaded blocks
            // stays mapped for the next loads instead of going back to the
            // driver at every synchronisation
            cudaMemPoolProps props;
            std::memset(&props, 0, sizeof(props));
            props.allocType = cudaMemAllocationTypePinned;
            props.location.type = cudaMemLocationTypeDevice;
            props.location.id = ctx->device;
            COW_CUDA(cudaMemPoolCreate(&ctx->pool, &props));
            uint64_t keep = ~(uint64_t)0;
            COW_CUDA(cudaMemPoolSetAttribute(ctx->pool, cudaMemPoolAttrReleaseThreshold, &keep));
        }
        if (!ctx->copy_stream) COW_CUDA(cudaStreamCreateWithFlags(&ctx->copy_stream, cudaStreamNonBlocking));
        if (!ctx->loaded) COW_CUDA(cudaEventCreateWithFlags(&ctx->loaded, cudaEventDisableTiming));
        // pinned host copies of every block's packed features (one buffer a
        // block, the tensors at the chunk offsets), taken once
        for (int32_t i = 0; i < nb; i++) {
            BlockHost &b = ctx->blocks[(size_t)i];
            if (b.host_feat) continue;
            const cudaError_t e = cudaMallocHost(&b.host_feat, (size_t)chunk_bytes(ctx, b));
            if (e != cudaSuccess) {
                cudaGetLastError();
                b.host_feat = nullptr;
                return fail(COW_ERR_OOM, "pinned host copy of block %d: %s", i, cudaGetErrorString(e));
            }
            for (int t = 0; t < 4; t++)
                COW_CUDA(cudaMemcpy((unsigned char *)b.host_feat + feature_offset(ctx, b, t), *tensor_slot(b, t),
                                    (size_t)tensor_bytes(ctx, b, t), cudaMemcpyDeviceToHost));
            b.dirty = false;
        }
        if (ctx->budget == 0) {
            // entering: every block is unloaded; each call loads what it needs
            ctx->resident_bytes = 0;
            for (const auto &b : ctx->blocks)
                if (b.resident) ctx->resident_bytes += feature_bytes(ctx, b);
            for (int32_t i = 0; i < nb; i++)
                if ((rc = evict_block(ctx, i)) != COW_OK) return rc;
        }
        ctx->budget = budget_bytes;
        while (ctx->resident_bytes > ctx->budget) {  // a smaller budget: unload least recently used first
            int32_t victim = -1;
            for (int32_t i = 0; i < nb; i++) {
                const BlockHost &b = ctx->blocks[(size_t)i];
                if (b.resident && (victim < 0 || b.last_use < ctx->blocks[(size_t)victim].last_use)) victim = i;
            }
            if ((rc = evict_block(ctx, victim)) != COW_OK) return rc;
        }
        COW_CUDA(cudaStreamSynchronize(ctx->copy_stream));
        return COW_OK;
    }
    if (ctx->budget == 0) return COW_OK;
    // leaving: load every block back, drop the host copies
    ctx->budget = 0;
    for (int32_t i = 0; i < nb; i++)
        if ((rc = upload_block(ctx, i)) != COW_OK) return rc;
    COW_CUDA(cudaStreamSynchronize(ctx->copy_stream));
    COW_CUDA(cudaMemPoolTrimTo(ctx->pool, 0));  // return what unloaded blocks left in the pool
    for (auto &b : ctx->blocks) {
        if (b.host_feat) cudaFreeHost(b.host_feat);
        b.host_feat = nullptr;
        b.dirty = false;
        b.use_ev.reset();
    }
    return COW_OK;
}

cow_status cow_get_residency(const cow_ctx *ctx, cow_residency *out) {
    if (!ctx || !out) return fail(COW_ERR_INVALID_ARG, "null argument");
    out->budget_bytes = ctx->budget;
    out->resident_bytes = ctx->resident_bytes;
    int32_t n = 0;
    for (const auto &b : ctx->blocks) n += b.resident ? 1 : 0;
    out->resident_blocks = n;
    out->uploads = ctx->n_uploads;
    out->upload_bytes = ctx->upload_bytes;
    out->evictions = ctx->n_evictions;
    out->evictions_waiting_last_call = ctx->n_evict_wait_last;
    return COW_OK;
}

cow_status cow_block_bytes(const cow_ctx *ctx, int32_t block, int64_t *out_bytes) {
    if (!ctx || !out_bytes) return fail(COW_ERR_INVALID_ARG, "null argument");
    if (block < 0 || block >= (int32_t)ctx->blocks.size()) return fail(COW_ERR_INVALID_ARG, "block out of range");
    *out_bytes = feature_bytes(ctx, ctx->blocks[(size_t)block]);
    return COW_OK;
}

namespace {

// Check a planning request: sizes, CSR offsets, ids, and every view's own
// blocks within the budget.
cow_status check_views(const int64_t *block_bytes, int32_t n_blocks, const int32_t *ids, const int32_t *ids_offsets,
                       int32_t n_views, int64_t budget_bytes) {
    if (ids_offsets[0] != 0) return fail(COW_ERR_INVALID_ARG, "ids_offsets[0] must be 0");
    for (int32_t i = 0; i < n_blocks; i++)
        if (block_bytes[i] < 0) return fail(COW_ERR_INVALID_ARG, "block %d: negative size", i);
    for (int32_t v = 0; v < n_views; v++) {
        if (ids_offsets[v + 1] < ids_offsets[v]) return fail(COW_ERR_INVALID_ARG, "ids_offsets must be non-decreasing");
        std::vector<char> seen((size_t)n_blocks, 0);
        int64_t need = 0;
        for (int32_t k = ids_offsets[v]; k < ids_offsets[v + 1]; k++) {
            if (!ids || ids[k] < 0 || ids[k] >= n_blocks)
                return fail(COW_ERR_INVALID_ARG, "view %d: block id out of range", v);
            if (!seen[(size_t)ids[k]]) need += block_bytes[ids[k]];
            seen[(size_t)ids[k]] = 1;
        }
        if (need > budget_bytes)
            return fail(COW_ERR_INVALID_ARG, "view %d needs %lld bytes, over the budget", v, (long long)need);
    }
    return COW_OK;
}

// The runtime's loading rule (ensure_resident) on block sizes alone, from
// the cold start cow_set_residency leaves: a view's call unloads the least
// recently used blocks it does not use (ties: lowest index) until its missing
// blocks fit, then loads them.
struct LruSim {
    const int64_t *bytes;
    int32_t nb;
    const int32_t *ids, *offs;
    int64_t budget;
    std::vector<char> res;
    std::vector<uint64_t> last;
    uint64_t clock = 0;
    int64_t used = 0;

    LruSim(const int64_t *b, int32_t n, const int32_t *i, const int32_t *o, int64_t bud)
        : bytes(b), nb(n), ids(i), offs(o), budget(bud), res((size_t)n, 0), last((size_t)n, 0) {}

    void reset() {
        std::fill(res.begin(), res.end(), 0);
        std::fill(last.begin(), last.end(), 0);
        clock = 0;
        used = 0;
    }
    // bytes view v would load now
    int64_t cost(int32_t v) const {
        std::vector<char> seen((size_t)nb, 0);
        int64_t m = 0;
        for (int32_t k = offs[v]; k < offs[v + 1]; k++)
            if (!seen[(size_t)ids[k]]) {
                seen[(size_t)ids[k]] = 1;
                if (!res[(size_t)ids[k]]) m += bytes[ids[k]];
            }
        return m;
    }
    // serve view v; returns the bytes it loaded
    int64_t apply(int32_t v) {
        std::vector<char> need((size_t)nb, 0);
        for (int32_t k = offs[v]; k < offs[v + 1]; k++) need[(size_t)ids[k]] = 1;
        int64_t missing = 0;
        for (int32_t i = 0; i < nb; i++)
            if (need[(size_t)i] && !res[(size_t)i]) missing += bytes[i];
        const uint64_t now = ++clock;
        for (int32_t i = 0; i < nb; i++)
            if (need[(size_t)i]) last[(size_t)i] = now;
        while (used + missing > budget) {
            int32_t victim = -1;
            for (int32_t i = 0; i < nb; i++) {
                if (!res[(size_t)i] || need[(size_t)i]) continue;
                if (victim < 0 || last[(size_t)i] < last[(size_t)victim]) victim = i;
            }
            if (victim < 0) break;
            res[(size_t)victim] = 0;
            used -= bytes[victim];
        }
        for (int32_t i = 0; i < nb; i++)
            if (need[(size_t)i] && !res[(size_t)i]) {
                res[(size_t)i] = 1;
                used += bytes[i];
            }
        return missing;
    }
    // bytes loaded serving `order` from a cold start
    int64_t total(const int32_t *order, int32_t n) {
        reset();
        int64_t s = 0;
        for (int32_t k = 0; k < n; k++) s += apply(order[k]);
        return s;
    }
};

}  // namespace

cow_status cow_plan_view_order(const int64_t *block_bytes, int32_t n_blocks, const int32_t *ids,
                               const int32_t *ids_offsets, int32_t n_views, int64_t budget_bytes, int32_t *out_order,
                               int64_t *out_upload_bytes, int64_t *out_upload_bytes_given) {
    g_last_error.clear();
    if (!block_bytes || n_blocks < 1 || !ids_offsets || n_views < 1 || budget_bytes < 1 || !out_order)
        return fail(COW_ERR_INVALID_ARG, "cow_plan_view_order: bad argument");
    cow_status rc = check_views(block_bytes, n_blocks, ids, ids_offsets, n_views, budget_bytes);
    if (rc != COW_OK) return rc;
    // greedy: next the view that loads the fewest bytes now (ties: lowest index)
    LruSim c(block_bytes, n_blocks, ids, ids_offsets, budget_bytes);
    std::vector<char> done((size_t)n_views, 0);
    int64_t planned = 0;
    for (int32_t s = 0; s < n_views; s++) {
        int32_t best = -1;
        int64_t best_cost = 0;
        for (int32_t v = 0; v < n_views; v++) {
            if (done[(size_t)v]) continue;
            const int64_t m = c.cost(v);
            if (best < 0 || m < best_cost) {
                best = v;
                best_cost = m;
            }
        }
        done[(size_t)best] = 1;
        out_order[s] = best;
        planned += c.apply(best);
    }
    if (out_upload_bytes) *out_upload_bytes = planned;
    if (out_upload_bytes_given) {
        std::vector<int32_t> given((size_t)n_views);
        for (int32_t v = 0; v < n_views; v++) given[(size_t)v] = v;
        *out_upload_bytes_given = c.total(given.data(), n_views);
    }
    return COW_OK;
}

cow_status cow_refine_view_order(const int64_t *block_bytes, int32_t n_blocks, const int32_t *ids,
                                 const int32_t *ids_offsets, int32_t n_views, int64_t budget_bytes, int32_t *io_order,
                                 int32_t max_evals, int64_t *out_upload_bytes) {
    g_last_error.clear();
    if (!block_bytes || n_blocks < 1 || !ids_offsets || n_views < 1 || budget_bytes < 1 || !io_order || max_evals < 1)
        return fail(COW_ERR_INVALID_ARG, "cow_refine_view_order: bad argument");
    cow_status rc = check_views(block_bytes, n_blocks, ids, ids_offsets, n_views, budget_bytes);
    if (rc != COW_OK) return rc;
    std::vector<char> seen((size_t)n_views, 0);
    for (int32_t k = 0; k < n_views; k++) {
        if (io_order[k] < 0 || io_order[k] >= n_views || seen[(size_t)io_order[k]])
            return fail(COW_ERR_INVALID_ARG, "io_order must be a permutation of 0 .. n_views-1");
        seen[(size_t)io_order[k]] = 1;
    }
    LruSim c(block_bytes, n_blocks, ids, ids_offsets, budget_bytes);
    std::vector<int32_t> cur(io_order, io_order + n_views), cand((size_t)n_views);
    int64_t best = c.total(cur.data(), n_views);
    int32_t evals = 1;
    // first improvement over single-view moves (view at i to place j), rescanned from the start after each
    bool improved = true;
    while (improved && evals < max_evals) {
        improved = false;
        for (int32_t i = 0; i < n_views && !improved && evals < max_evals; i++)
            for (int32_t j = 0; j < n_views && !improved && evals < max_evals; j++) {
                if (j == i) continue;
                cand = cur;
                const int32_t v = cand[(size_t)i];
                cand.erase(cand.begin() + i);
                cand.insert(cand.begin() + j, v);
                const int64_t t = c.total(cand.data(), n_views);
                evals++;
                if (t < best) {
                    best = t;
                    cur.swap(cand);
                    improved = true;
                }
            }
    }
    std::copy(cur.begin(), cur.end(), io_order);
    if (out_upload_bytes) *out_upload_bytes = best;
    return COW_OK;
}

cow_status cow_set_tile_order(cow_ctx *ctx, int32_t strip_tiles) {
    if (!ctx) return fail(COW_ERR_INVALID_ARG, "null context");
    if (strip_tiles < 0 || strip_tiles > 4096) return fail(COW_ERR_INVALID_ARG, "strip_tiles must be in [0, 4096]");
    ctx->tile_strip = strip_tiles;
    return COW_OK;
}

cow_status cow_tune_schedule(cow_ctx *ctx, const cow_camera *cams, int32_t n_views, const int32_t *ids,
                             const int32_t *ids_offsets, const float *mlp, float ert_eps, uint32_t flags,
                             float *out_rgb, int32_t reps, void *stream, int32_t *out_schedule,
                             int32_t *out_strip, float *out_ms) {
    g_last_error.clear();
    if (!ctx || !out_rgb || reps < 1) return fail(COW_ERR_INVALID_ARG, "cow_tune_schedule: bad argument");
    if (!is_device_ptr(out_rgb)) return fail(COW_ERR_INVALID_ARG, "cow_tune_schedule: out_rgb must be device memory");
    DeviceGuard dg(ctx->device);
    cudaStream_t st = (cudaStream_t)stream;
    static const int kScheds[] = {COW_SCHED_THREAD_CONST, COW_SCHED_THREAD, COW_SCHED_WARP};
    static const int kStrips[] = {0, 2, 4};
    const int s0 = ctx->schedule, t0 = ctx->tile_strip;
    cudaEvent_t e0, e1;
    COW_CUDA(cudaEventCreate(&e0));
    COW_CUDA(cudaEventCreate(&e1));
    float best = 3.0e38f;
    int best_s = s0, best_t = t0;
    cow_status rc = COW_OK;
    for (int sc : kScheds) {
        for (int tr : kStrips) {
            ctx->schedule = sc;
            ctx->tile_strip = tr;
            rc = cow_render(ctx, cams, n_views, ids, ids_offsets, mlp, ert_eps, flags, out_rgb, nullptr, nullptr, stream);
            if (rc != COW_OK) break;
            cudaEventRecord(e0, st);
            for (int r = 0; r < reps && rc == COW_OK; r++)
                rc = cow_render(ctx, cams, n_views, ids, ids_offsets, mlp, ert_eps, flags, out_rgb, nullptr, nullptr,
                                stream);
            cudaEventRecord(e1, st);
            if (rc != COW_OK) break;
            if (cudaEventSynchronize(e1) != cudaSuccess) {
                rc = fail(COW_ERR_CUDA, "cow_tune_schedule: synchronisation failed");
                break;
            }
            float ms = 0.f;
            cudaEventElapsedTime(&ms, e0, e1);
            ms /= (float)reps;
            if (ms < best) {
                best = ms;
                best_s = sc;
                best_t = tr;
            }
        }
        if (rc != COW_OK) break;
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    ctx->schedule = rc == COW_OK ? best_s : s0;
    ctx->tile_strip = rc == COW_OK ? best_t : t0;
    if (rc != COW_OK) return rc;
    if (out_schedule) *out_schedule = best_s;
    if (out_strip) *out_strip = best_t;
    if (out_ms) *out_ms = best;
    return COW_OK;
}

cow_status cow_set_ray_order(cow_ctx *ctx, int32_t mode) {
    g_last_error.clear();
    if (!ctx) return fail(COW_ERR_INVALID_ARG, "null context");
    if (mode != COW_RAY_ORDER_GIVEN && mode != COW_RAY_ORDER_COHERENT)
        return fail(COW_ERR_INVALID_ARG, "unknown ray order %d", mode);
    ctx->ray_order = mode;
    return COW_OK;
}

cow_status cow_set_schedule(cow_ctx *ctx, int32_t schedule) {
    if (!ctx) return fail(COW_ERR_INVALID_ARG, "null context");
    if (schedule != COW_SCHED_WARP && schedule != COW_SCHED_THREAD && schedule != COW_SCHED_THREAD_CONST)
        return fail(COW_ERR_INVALID_ARG, "unknown schedule %d", schedule);
    ctx->schedule = schedule;
    return COW_OK;
}

static_assert(COW_TEST_SKIP_RECORD_COPY == cow::kTestSkipRecordCopy, "test flag values");

cow_status cow_set_test_hooks(cow_ctx *ctx, uint32_t flags, uint32_t wait_polls) {
    g_last_error.clear();
    if (!ctx) return fail(COW_ERR_INVALID_ARG, "null context");
    if (flags & ~(uint32_t)COW_TEST_SKIP_RECORD_COPY) return fail(COW_ERR_INVALID_ARG, "unknown test flags 0x%x", flags);
    ctx->test_flags = flags;
    ctx->wait_polls = wait_polls;
    return COW_OK;
}

cow_status cow_sync_check(cow_ctx *ctx, void *stream) {
    if (!ctx) return fail(COW_ERR_INVALID_ARG, "null context");
    DeviceGuard dg(ctx->device);
    cudaStream_t st = (cudaStream_t)stream;
    COW_CUDA(cudaStreamSynchronize(st));
    unsigned err = 0;
    COW_CUDA(cudaMemcpy(&err, ctx->d_err, sizeof(err), cudaMemcpyDeviceToHost));
    if (err) {
        COW_CUDA(cudaMemset(ctx->d_err, 0, sizeof(unsigned)));
        if (err & cow::kErrTimeout) return fail(COW_ERR_TIMEOUT, "a bounded device-side wait ran out (error word 0x%x)", err);
        return fail(COW_ERR_DEVICE_ASSERT, "a kernel range check fired (error word 0x%x)", err);
    }
    return COW_OK;
}

cow_status cow_export_occupancy(const cow_ctx *ctx, int32_t block, uint32_t *out_bits, int64_t n_words) {
    if (!ctx || !out_bits) return fail(COW_ERR_INVALID_ARG, "null argument");
    if (block < 0 || block >= (int32_t)ctx->blocks.size()) return fail(COW_ERR_INVALID_ARG, "block out of range");
    const BlockHost &b = ctx->blocks[(size_t)block];
    if (n_words < b.occ_words) return fail(COW_ERR_INVALID_ARG, "need %lld words", (long long)b.occ_words);
    DeviceGuard dg(ctx->device);
    COW_CUDA(cudaMemcpy(out_bits, b.occ, (size_t)b.occ_words * 4, cudaMemcpyDeviceToHost));
    return COW_OK;
}

cow_status cow_export_occupancy_coarse(const cow_ctx *ctx, int32_t block, uint32_t *out_bits, int64_t n_words) {
    if (!ctx || !out_bits) return fail(COW_ERR_INVALID_ARG, "null argument");
    if (block < 0 || block >= (int32_t)ctx->blocks.size()) return fail(COW_ERR_INVALID_ARG, "block out of range");
    const BlockHost &b = ctx->blocks[(size_t)block];
    if (n_words < b.occ2_words) return fail(COW_ERR_INVALID_ARG, "need %lld words", (long long)b.occ2_words);
    DeviceGuard dg(ctx->device);
    COW_CUDA(cudaMemcpy(out_bits, b.occ2, (size_t)b.occ2_words * 4, cudaMemcpyDeviceToHost));
    return COW_OK;
}

cow_status cow_export_packed(const cow_ctx *ctx, int32_t block, int32_t tensor, void *out, int64_t nbytes,
                             int32_t *out_scale_exp) {
    if (!ctx || !out) return fail(COW_ERR_INVALID_ARG, "null argument");
    const int max_tensor = ctx->dtype == COW_FP8_BF16D ? 4 : 3;
    if (block < 0 || block >= (int32_t)ctx->blocks.size() || tensor < 0 || tensor > max_tensor)
        return fail(COW_ERR_INVALID_ARG, "block or tensor out of range");
    const BlockHost &b = ctx->blocks[(size_t)block];
    if ((tensor == 0 || tensor == 4) && b.Nb > 0)
        return fail(COW_ERR_UNSUPPORTED, "a brick-sparse grid holds no dense copy to export");
    const int64_t nv = tensor == 0 || tensor == 4 ? (int64_t)b.R * b.R * b.R : (int64_t)b.P * b.P;
    // tensor 4: the BF16 channel 0 of the FP8 format's grid (one value a vertex)
    const int tdt = tensor == 4 ? COW_BF16 : tensor_dtype(ctx->dtype, tensor);
    const int64_t nch = tensor == 4 ? 1 : cow::kNch;
    const int64_t need = nv * nch * elem_bytes(tdt);
    if (nbytes < need) return fail(COW_ERR_INVALID_ARG, "need %lld bytes", (long long)need);
    DeviceGuard dg(ctx->device);
    // an unloaded block is read from its pinned host copy (after any
    // write-back still queued on the copy stream)
    if (!b.resident && ctx->copy_stream) COW_CUDA(cudaStreamSynchronize(ctx->copy_stream));
    const int tslot = tensor == 4 ? 0 : tensor;
    const void *src = !b.resident ? (const void *)((const unsigned char *)b.host_feat + feature_offset(ctx, b, tslot))
                                  : tensor == 0 || tensor == 4 ? b.grid : b.planes[tensor - 1];
    if (tensor == 4) src = (const unsigned char *)src + grid_main_bytes(ctx, b);
    if (ctx->dtype == COW_FP32) {
        COW_CUDA(cudaMemcpy(out, src, (size_t)need, cudaMemcpyDefault));
    } else {
        // pair layout on the device: keep the first vertex of every pair (the
        // first texel of a quad, the first corner of a density octet)
        const int64_t pe = tensor == 4 ? 16 : packed_elem_bytes(ctx->dtype), ve = nch * elem_bytes(tdt);
        std::vector<unsigned char> raw((size_t)(nv * pe));
        COW_CUDA(cudaMemcpy(raw.data(), src, raw.size(), cudaMemcpyDefault));
        for (int64_t i = 0; i < nv; i++) std::memcpy((unsigned char *)out + i * ve, raw.data() + i * pe, (size_t)ve);
    }
    if (out_scale_exp)
        for (int k = 0; k < 8; k++) out_scale_exp[k] = tensor == 4 ? 0 : b.scale_exp[tensor][k];
    return COW_OK;
}

}  // extern "C"

// ---------------------------------------------------------------------------
// Allocation-free backward.
//
// Some callers cannot allocate device memory once they are running: a
// trainer or viewer that works inside a fixed device-memory budget (its
// memory pool is frozen after start-up), or a steady-state loop that must not
// pay for cudaMalloc / cudaFree (cudaFree also synchronises the device).
// cow_render_backward_noalloc serves them: it computes exactly what
// cow_render_backward computes, but its scratch -- the per-CTA rows of the
// MLP weight gradient, the per-ray dL/dC_d, dL/dF and the per-block gradient
// pointer table -- lives in the file-scope array below instead of context
// buffers, so the call itself allocates nothing.  The pointer table is
// written on the device by a one-CTA kernel that receives the call's
// gradient pointers as launch parameters, so no device work reads host
// memory after the call returns.
//
// Limits: at most kNoAllocMaxRays rays and kNoAllocMaxBlocks blocks per call
// (3 MiB of device memory, held by every GPU that loads the library until the
// process exits).  All calls on a device share the array: every call rewrites
// the parts it reads before reading them, so nothing has to start at zero,
// but calls that overlap on the GPU (different streams, or different
// contexts on one device) race on it and must be ordered by the caller.

namespace {

constexpr int64_t kNoAllocMaxRays = 65536;
constexpr int32_t kNoAllocMaxBlocks = 1024;
// one MLP-gradient row per backward CTA: backward_rows(kNoAllocMaxRays) rows
constexpr int64_t kNaRows = (kNoAllocMaxRays + cow::kBwdCtaThreads - 1) / cow::kBwdCtaThreads;
constexpr size_t kNaRowsBytes = ((size_t)kNaRows * cow::kMlpParams * sizeof(float) + 255) / 256 * 256;
constexpr size_t kNaGcfBytes = (size_t)kNoAllocMaxRays * 8 * sizeof(float);     // 2 MiB
constexpr size_t kNaPtrBytes = (size_t)kNoAllocMaxBlocks * 4 * sizeof(float *);  // 32 KiB
constexpr size_t kNaTotalBytes = kNaRowsBytes + kNaGcfBytes + kNaPtrBytes;
static_assert(kNaRowsBytes % 256 == 0 && kNaGcfBytes % 256 == 0 && kNaPtrBytes % 256 == 0,
              "scratch sections must keep 256-byte alignment");
static_assert(kNaRowsBytes >= (size_t)kNaRows * cow::kMlpParams * sizeof(float), "row section holds every row");

// In host code this name is only a host-side handle, not a device address;
// the device address comes from cudaGetSymbolAddress below.
static __device__ __align__(256) unsigned char g_noalloc_scratch[kNaTotalBytes];

// The gradient pointers of one call's blocks, passed by value.
struct NaPtrFill {
    int32_t n;
    int32_t id[cow::kMaxRayIds];
    float *p[cow::kMaxRayIds][4];  // grid, planes xy, xz, yz (entries may be null)
};

// table[id] = grid gradient, table[nb + 3 id + k] = plane k gradient: the
// layout the backward kernels index by block id.
__global__ void k_noalloc_fill_ptrs(float **table, int32_t nb, const __grid_constant__ NaPtrFill f) {
    const int k = threadIdx.x;
    if (k >= f.n) return;
    const int id = f.id[k];
    table[id] = f.p[k][0];
    for (int q = 0; q < 3; q++) table[nb + 3 * id + q] = f.p[k][1 + q];
}

constexpr int kMaxDevices = 64;
std::mutex g_noalloc_mu;
void *g_noalloc_addr[kMaxDevices] = {nullptr};

// Device address of the scratch array on the current device, looked up once
// per device (the first call on a device does this; make that first call
// before any stream capture).
cow_status noalloc_scratch(int device, unsigned char **out) {
    if (device < 0 || device >= kMaxDevices) return fail(COW_ERR_UNSUPPORTED, "device index %d too large", device);
    std::lock_guard<std::mutex> lock(g_noalloc_mu);
    if (!g_noalloc_addr[device]) {
        void *p = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess || !p)
            return fail(COW_ERR_CUDA, "cudaGetSymbolAddress of the backward scratch failed: %s", cudaGetErrorString(e));
        g_noalloc_addr[device] = p;
    }
    *out = (unsigned char *)g_noalloc_addr[device];
    return COW_OK;
}

}  // namespace

extern "C" cow_status cow_render_backward_noalloc(cow_ctx *ctx, const float *o, const float *d, int64_t n_rays,
                                                  const int32_t *ids, int32_t n_ids, const float *mlp,
                                                  float ert_eps, const float *aux, const float *dL_drgb,
                                                  float *const *grad_grid, float *const *grad_planes,
                                                  float *grad_mlp, void *stream) {
    g_last_error.clear();
    if (ctx && n_rays == 0) return COW_OK;  // an empty batch (its arrays may be NULL)
    if (!ctx || !o || !d || n_rays < 0 || !ids || !mlp || !aux || !dL_drgb || !grad_grid || !grad_planes || !grad_mlp)
        return fail(COW_ERR_INVALID_ARG, "cow_render_backward_noalloc: null argument");
    if (n_rays > kNoAllocMaxRays || cow::backward_rows(n_rays) > kNaRows)
        return fail(COW_ERR_INVALID_ARG, "cow_render_backward_noalloc: %lld rays exceed its maximum of %lld per call",
                    (long long)n_rays, (long long)kNoAllocMaxRays);
    const int32_t nb = (int32_t)ctx->blocks.size();
    if (nb > kNoAllocMaxBlocks)
        return fail(COW_ERR_INVALID_ARG, "cow_render_backward_noalloc: %d blocks exceed its maximum of %d", nb,
                    kNoAllocMaxBlocks);
    if (n_ids < 1 || n_ids > cow::kMaxRayIds) return fail(COW_ERR_INVALID_ARG, "n_ids must be in [1, %d]", cow::kMaxRayIds);
    if (!(ert_eps >= 0.0f && ert_eps < 1.0f)) return fail(COW_ERR_INVALID_ARG, "ert_eps must be in [0, 1)");
    for (int32_t k = 0; k < n_ids; k++)
        if (ids[k] < 0 || ids[k] >= nb) return fail(COW_ERR_INVALID_ARG, "block id %d out of range", ids[k]);
    for (int32_t k = 0; k < n_ids; k++)
        if (!ctx->blocks[(size_t)ids[k]].resident)
            return fail(COW_ERR_INVALID_ARG, "block %d is unloaded: the no-allocation entry point loads no blocks (render "
                        "the rays with cow_render_rays first)", ids[k]);
    for (const void *q : {(const void *)o, (const void *)d, (const void *)aux, (const void *)dL_drgb, (const void *)grad_mlp, (const void *)mlp})
        if (!is_device_ptr(q)) return fail(COW_ERR_INVALID_ARG, "backward arrays and the MLP must be device memory");
    if (((uintptr_t)aux & 15u)) return fail(COW_ERR_INVALID_ARG, "aux must be 16-byte aligned");
    for (int32_t i = 0; i < nb; i++)
        for (int k = 0; k < 4; k++) {
            const float *q = k == 0 ? grad_grid[i] : grad_planes[3 * i + k - 1];
            if (q && (((uintptr_t)q & 15u) || !is_device_ptr(q)))
                return fail(COW_ERR_INVALID_ARG, "block %d: gradient arrays must be 16-byte aligned device memory", i);
        }
    NaPtrFill fill;
    std::memset(&fill, 0, sizeof(fill));
    fill.n = n_ids;
    for (int32_t k = 0; k < n_ids; k++) {
        const int32_t id = ids[k];
        fill.id[k] = id;
        fill.p[k][0] = grad_grid[id];
        for (int q = 0; q < 3; q++) fill.p[k][1 + q] = grad_planes[3 * id + q];
    }
    DeviceGuard dg(ctx->device);
    unsigned char *scratch = nullptr;
    cow_status rc = noalloc_scratch(ctx->device, &scratch);
    if (rc != COW_OK) return rc;
    float *rows = (float *)scratch;
    float *gcf = (float *)(scratch + kNaRowsBytes);
    float **dptrs = (float **)(scratch + kNaRowsBytes + kNaGcfBytes);
    cudaStream_t st = (cudaStream_t)stream;
    k_noalloc_fill_ptrs<<<1, cow::kMaxRayIds, 0, st>>>(dptrs, nb, fill);
    COW_CUDA(cudaGetLastError());
    cow::BwdArgs a;
    std::memset(&a, 0, sizeof(a));
    a.dtype = kernel_dtype(ctx);
    a.mlp = mlp;
    a.ert_eps = ert_eps;
    a.ray_o = o;
    a.ray_d = d;
    a.n_rays = n_rays;
    a.aux = aux;
    a.dL_drgb = dL_drgb;
    a.grad_grid = dptrs;
    a.grad_planes = dptrs + nb;
    a.grad_mlp = grad_mlp;
    a.partials = rows;
    a.gcf = gcf;
    a.err = ctx->d_err;
    cow::RayRecs rr;
    make_ray_recs(ctx, ids, n_ids, rr);
    COW_CUDA(cow::launch_backward_rays(a, rr, st));
    return note_use_impl(ctx, ids, n_ids, st);
}
