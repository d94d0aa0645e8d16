// scene_io.cu -- save and load a packed scene (the baked blocks as the
// context holds them: packed features in the storage format, occupancy
// levels, scales, brick tables), so a viewer can start from the baked
// assets without the FP32 masters or a re-pack.  The file is a fixed binary
// header and block table, a JSON manifest of the same facts for other tools,
// then the raw arrays.
#include <cmath>
#include <cstdio>
#include <cstring>
#include <string>
#include <vector>

#include "cow_internal.h"

using namespace cowi;

namespace {

constexpr char kMagic[8] = {'C', 'O', 'W', 'S', 'C', 'N', '0', '1'};
constexpr uint32_t kVersion = 1;
constexpr int kSections = 8;  // grid (+ density octets), planes xy / xz / yz, occ, occ2, brick table, brick list

struct FileHeader {
    char magic[8];
    uint32_t version;
    int32_t n_blocks;
    int32_t dtype, bricks, occ_cell;
    float occ_thresh;
    uint64_t json_bytes;
};

struct FileBlock {
    float lo[3], hi[3];
    int32_t lod, parent, R, P, unb, Nb, n_bricks, pad_;
    double ztop;
    int32_t scale_exp[4][8];
    uint64_t off[kSections], bytes[kSections];
};

static_assert(sizeof(FileHeader) == 40 && sizeof(FileBlock) == 320, "the packed scene file layout is fixed");

struct FileCloser {
    FILE *f;
    ~FileCloser() {
        if (f) fclose(f);
    }
};

// the device (or pinned host) array of section k of a block and its bytes
const void *section_src(const cow_ctx *c, const BlockHost &b, int k, int64_t *bytes, int64_t t_bytes[4],
                        int64_t t_off[4]) {
    if (k < 4) {
        *bytes = t_bytes[k];
        if (!b.resident) return (const unsigned char *)b.host_feat + t_off[k];
        return k == 0 ? b.grid : b.planes[k - 1];
    }
    if (k == 4) {
        *bytes = b.occ_words * 4;
        return b.occ;
    }
    if (k == 5) {
        *bytes = b.occ2_words * 4;
        return b.occ2;
    }
    if (k == 6) {
        *bytes = b.Nb > 0 ? (int64_t)b.Nb * b.Nb * b.Nb * 4 : 0;
        return b.brick_tab;
    }
    *bytes = b.Nb > 0 ? (int64_t)b.n_bricks * 4 : 0;
    return b.brick_list;
}

// The coarse level is the OR of the fine cells of each group; with bricks, the
// table and the list are inverse of each other, and every coarse cell with a
// set bit has a stored brick.  sec: the block's occ, occ2, brick table and
// brick list as read from the file.
bool occupancy_consistent(const BlockHost &b, int Nc, int Nc2, const std::vector<unsigned char> sec[4]) {
    const uint32_t *occ = (const uint32_t *)sec[0].data();
    const uint32_t *occ2 = (const uint32_t *)sec[1].data();
    std::vector<uint32_t> coarse(((size_t)Nc2 * Nc2 * Nc2 + 31) / 32, 0u);
    for (int z = 0; z < Nc; z++)
        for (int y = 0; y < Nc; y++)
            for (int x = 0; x < Nc; x++) {
                const int64_t ci = ((int64_t)z * Nc + y) * Nc + x;
                if (!((occ[ci >> 5] >> (ci & 31)) & 1u)) continue;
                const int64_t c2 = ((int64_t)(z >> cow::kOccGroupLog2) * Nc2 + (y >> cow::kOccGroupLog2)) * Nc2 +
                                   (x >> cow::kOccGroupLog2);
                coarse[(size_t)(c2 >> 5)] |= 1u << (c2 & 31);
            }
    if (sec[1].size() != coarse.size() * 4 || std::memcmp(occ2, coarse.data(), sec[1].size()) != 0) return false;
    if (b.Nb == 0) return true;
    const int64_t n3 = (int64_t)b.Nb * b.Nb * b.Nb;
    const int32_t *tab = (const int32_t *)sec[2].data();
    const int32_t *list = (const int32_t *)sec[3].data();
    for (int32_t s = 0; s < b.n_bricks; s++)
        if (list[s] < 0 || list[s] >= n3 || tab[list[s]] != s) return false;
    for (int64_t k = 0; k < n3; k++) {
        const bool set = (coarse[(size_t)(k >> 5)] >> (k & 31)) & 1u;
        if (tab[k] < -1 || tab[k] >= b.n_bricks || (set && tab[k] < 0)) return false;
    }
    return true;
}

}  // namespace

extern "C" {

cow_status cow_save_scene(const cow_ctx *ctx, const char *path) {
    g_last_error.clear();
    COW_NVTX("cow_save_scene");
    if (!ctx || !path) return fail(COW_ERR_INVALID_ARG, "cow_save_scene: null argument");
    DeviceGuard dg(ctx->device);
    COW_CUDA(cudaDeviceSynchronize());  // pending work (and write-backs of unloaded blocks) first
    const int32_t nb = (int32_t)ctx->blocks.size();
    std::vector<FileBlock> table((size_t)nb);
    std::string json = "{\"format\": \"cow packed scene\", \"version\": 1, \"dtype\": " + std::to_string(ctx->dtype) +
                       ", \"bricks\": " + std::to_string(ctx->bricks ? 1 : 0) +
                       ", \"occ_cell\": " + std::to_string(ctx->occ_cell) + ", \"blocks\": [";
    std::vector<std::vector<int64_t>> sb((size_t)nb);
    uint64_t off = 0;
    for (int32_t i = 0; i < nb; i++) {
        const BlockHost &b = ctx->blocks[(size_t)i];
        FileBlock &fb = table[(size_t)i];
        std::memset(&fb, 0, sizeof(fb));
        for (int a = 0; a < 3; a++) {
            fb.lo[a] = b.lo[a];
            fb.hi[a] = b.hi[a];
        }
        fb.lod = b.lod;
        fb.parent = b.parent;
        fb.R = b.R;
        fb.P = b.P;
        fb.unb = b.unb;
        fb.Nb = b.Nb;
        fb.n_bricks = b.n_bricks;
        fb.ztop = b.ztop;
        std::memcpy(fb.scale_exp, b.scale_exp, sizeof(fb.scale_exp));
        int64_t tb[4], to[4];
        for (int t = 0; t < 4; t++) {
            tb[t] = block_tensor_bytes(ctx, b, t);
            to[t] = block_feature_offset(ctx, b, t);
        }
        for (int k = 0; k < kSections; k++) {
            int64_t by = 0;
            section_src(ctx, b, k, &by, tb, to);
            fb.off[k] = off;
            fb.bytes[k] = (uint64_t)by;
            off += ((uint64_t)by + 255) & ~(uint64_t)255;
        }
        char buf[256];
        std::snprintf(buf, sizeof(buf), "%s{\"lo\": [%.9g, %.9g, %.9g], \"hi\": [%.9g, %.9g, %.9g], \"lod\": %d, \"R\": %d, \"P\": %d, \"bricks_stored\": %d}",
                      i ? ", " : "", b.lo[0], b.lo[1], b.lo[2], b.hi[0], b.hi[1], b.hi[2], b.lod, b.R, b.P, b.n_bricks);
        json += buf;
    }
    json += "]}\n";
    FILE *f = std::fopen(path, "wb");
    if (!f) return fail(COW_ERR_INVALID_ARG, "cow_save_scene: cannot open %s for writing", path);
    FileCloser fc{f};
    FileHeader h;
    std::memset(&h, 0, sizeof(h));
    std::memcpy(h.magic, kMagic, 8);
    h.version = kVersion;
    h.n_blocks = nb;
    h.dtype = ctx->dtype;
    h.bricks = ctx->bricks ? 1 : 0;
    h.occ_cell = ctx->occ_cell;
    h.occ_thresh = ctx->occ_thresh;
    h.json_bytes = json.size();
    if (std::fwrite(&h, sizeof(h), 1, f) != 1 || std::fwrite(table.data(), sizeof(FileBlock), table.size(), f) != table.size() ||
        std::fwrite(json.data(), 1, json.size(), f) != json.size())
        return fail(COW_ERR_INVALID_ARG, "cow_save_scene: write to %s failed", path);
    const long data0 = (std::ftell(f) + 255) & ~255L;
    std::vector<unsigned char> host;
    for (int32_t i = 0; i < nb; i++) {
        const BlockHost &b = ctx->blocks[(size_t)i];
        int64_t tb[4], to[4];
        for (int t = 0; t < 4; t++) {
            tb[t] = block_tensor_bytes(ctx, b, t);
            to[t] = block_feature_offset(ctx, b, t);
        }
        for (int k = 0; k < kSections; k++) {
            int64_t by = 0;
            const void *src = section_src(ctx, b, k, &by, tb, to);
            if (by == 0) continue;
            host.resize((size_t)by);
            COW_CUDA(cudaMemcpy(host.data(), src, (size_t)by, cudaMemcpyDefault));
            if (std::fseek(f, data0 + (long)table[(size_t)i].off[k], SEEK_SET) != 0 ||
                std::fwrite(host.data(), 1, (size_t)by, f) != (size_t)by)
                return fail(COW_ERR_INVALID_ARG, "cow_save_scene: write to %s failed", path);
        }
    }
    if (std::fflush(f) != 0) return fail(COW_ERR_INVALID_ARG, "cow_save_scene: write to %s failed", path);
    return COW_OK;
}

cow_status cow_load_scene(cow_ctx **out, const char *path, void *stream) {
    g_last_error.clear();
    COW_NVTX("cow_load_scene");
    if (!out || !path) return fail(COW_ERR_INVALID_ARG, "cow_load_scene: null argument");
    *out = nullptr;
    FILE *f = std::fopen(path, "rb");
    if (!f) return fail(COW_ERR_INVALID_ARG, "cow_load_scene: cannot open %s", path);
    FileCloser fc{f};
    FileHeader h;
    if (std::fread(&h, sizeof(h), 1, f) != 1 || std::memcmp(h.magic, kMagic, 8) != 0 || h.version != kVersion)
        return fail(COW_ERR_INVALID_ARG, "cow_load_scene: %s is not a packed scene of this version", path);
    if (h.n_blocks < 1 || h.n_blocks > (1 << 20) || h.dtype < 0 || h.dtype > 5 || h.occ_cell < 1 || h.occ_cell > 4096 ||
        h.json_bytes > ((uint64_t)1 << 30))
        return fail(COW_ERR_INVALID_ARG, "cow_load_scene: bad header in %s", path);
    std::vector<FileBlock> table((size_t)h.n_blocks);
    if (std::fread(table.data(), sizeof(FileBlock), table.size(), f) != table.size())
        return fail(COW_ERR_INVALID_ARG, "cow_load_scene: truncated block table in %s", path);
    const long data0 = (long)((sizeof(h) + table.size() * sizeof(FileBlock) + h.json_bytes + 255) & ~(uint64_t)255);
    cow_ctx *c = new cow_ctx();
    auto bail = [&](cow_status s) {
        destroy_context(c);
        return s;
    };
    if (cudaGetDevice(&c->device) != cudaSuccess) {
        delete c;
        return fail(COW_ERR_CUDA, "no CUDA device");
    }
    c->dtype = h.dtype;
    c->bricks = h.bricks != 0;
    c->occ_cell = h.occ_cell;
    c->occ_thresh = h.occ_thresh;
    c->blocks.resize(table.size());
    cudaStream_t st = (cudaStream_t)stream;
    cudaError_t e = cudaMalloc((void **)&c->d_err, sizeof(unsigned));
    if (e == cudaSuccess) e = cudaMalloc((void **)&c->d_mlp, 512 * sizeof(float));
    if (e == cudaSuccess) e = cudaMemset(c->d_err, 0, sizeof(unsigned));
    if (e != cudaSuccess) return bail(fail(COW_ERR_OOM, "cow_load_scene: %s", cudaGetErrorString(e)));
    std::vector<unsigned char> host;
    std::vector<unsigned char> sec[4];  // host copies of sections 4-7: occ, occ2, brick table, brick list
    for (size_t i = 0; i < table.size(); i++) {
        for (auto &v : sec) v.clear();
        const FileBlock &fb = table[i];
        BlockHost &b = c->blocks[i];
        bool box_ok = fb.lod >= 1;
        for (int a = 0; a < 3; a++) box_ok = box_ok && std::isfinite(fb.lo[a]) && std::isfinite(fb.hi[a]) && fb.lo[a] < fb.hi[a];
        if (fb.R < 2 || fb.P < 2 || fb.R > 1024 || fb.P > 16384 || fb.parent < -1 || fb.parent >= h.n_blocks ||
            fb.parent == (int32_t)i || fb.Nb < 0 || fb.n_bricks < 0 || (fb.Nb > 0) != c->bricks || !box_ok)
            return bail(fail(COW_ERR_INVALID_ARG, "cow_load_scene: bad block %zu in %s", i, path));
        for (int a = 0; a < 3; a++) {
            b.lo[a] = fb.lo[a];
            b.hi[a] = fb.hi[a];
        }
        b.lod = fb.lod;
        b.parent = fb.parent;
        b.R = fb.R;
        b.P = fb.P;
        b.unb = fb.unb;
        b.Nb = fb.Nb;
        b.n_bricks = fb.n_bricks;
        b.ztop = fb.ztop;
        std::memcpy(b.scale_exp, fb.scale_exp, sizeof(fb.scale_exp));
        const int Nc = (b.R - 1 + c->occ_cell - 1) / c->occ_cell;
        const int Nc2 = (Nc + cow::kOccGroup - 1) / cow::kOccGroup;
        if (c->bricks && (c->occ_cell != 4 || b.Nb != Nc2 || (int64_t)b.n_bricks > (int64_t)Nc2 * Nc2 * Nc2))
            return bail(fail(COW_ERR_INVALID_ARG, "cow_load_scene: bad brick counts for block %zu in %s", i, path));
        b.occ_words = ((int64_t)Nc * Nc * Nc + 31) / 32;
        b.occ2_words = ((int64_t)Nc2 * Nc2 * Nc2 + 31) / 32;
        const int64_t want[kSections] = {block_tensor_bytes(c, b, 0), block_tensor_bytes(c, b, 1),
                                         block_tensor_bytes(c, b, 2), block_tensor_bytes(c, b, 3), b.occ_words * 4,
                                         b.occ2_words * 4, b.Nb > 0 ? (int64_t)b.Nb * b.Nb * b.Nb * 4 : 0,
                                         b.Nb > 0 ? (int64_t)b.n_bricks * 4 : 0};
        void **dst[kSections] = {&b.grid, &b.planes[0], &b.planes[1], &b.planes[2], (void **)&b.occ,
                                 (void **)&b.occ2, (void **)&b.brick_tab, (void **)&b.brick_list};
        for (int k = 0; k < kSections; k++) {
            if ((int64_t)fb.bytes[k] != want[k])
                return bail(fail(COW_ERR_INVALID_ARG, "cow_load_scene: block %zu section %d has %llu bytes, expected %lld",
                                 i, k, (unsigned long long)fb.bytes[k], (long long)want[k]));
            const size_t alloc = (size_t)std::max<int64_t>(want[k], k == 7 && b.Nb > 0 ? 4 : 0);
            if (alloc == 0) continue;
            e = cudaMalloc(dst[k], alloc);
            if (e != cudaSuccess) return bail(fail(COW_ERR_OOM, "cow_load_scene: %s", cudaGetErrorString(e)));
            if (want[k] == 0) continue;
            host.resize((size_t)want[k]);
            if (std::fseek(f, data0 + (long)fb.off[k], SEEK_SET) != 0 ||
                std::fread(host.data(), 1, (size_t)want[k], f) != (size_t)want[k])
                return bail(fail(COW_ERR_INVALID_ARG, "cow_load_scene: truncated data in %s", path));
            e = cudaMemcpy(*dst[k], host.data(), (size_t)want[k], cudaMemcpyHostToDevice);
            if (e != cudaSuccess) return bail(fail(COW_ERR_CUDA, "cow_load_scene: %s", cudaGetErrorString(e)));
            if (k >= 4) sec[k - 4].assign(host.begin(), host.end());
        }
        // the occupancy levels and the brick table must describe one another:
        // the kernels skip a coarse cell whose bit is clear without reading its
        // fine cells, and read the brick of every occupied cell without testing
        // its slot, so a file that breaks this is refused rather than rendered
        if (!occupancy_consistent(b, Nc, Nc2, sec))
            return bail(fail(COW_ERR_INVALID_ARG, "cow_load_scene: block %zu in %s has inconsistent occupancy or bricks",
                             i, path));
        e = cudaMalloc((void **)&b.scale, 32 * sizeof(float));
        if (e != cudaSuccess) return bail(fail(COW_ERR_OOM, "cow_load_scene: %s", cudaGetErrorString(e)));
        float scale_h[32];
        for (int t = 0; t < 4; t++)
            for (int k = 0; k < 8; k++) scale_h[8 * t + k] = std::ldexp(1.0f, b.scale_exp[t][k]);
        e = cudaMemcpy(b.scale, scale_h, sizeof(scale_h), cudaMemcpyHostToDevice);
        if (e != cudaSuccess) return bail(fail(COW_ERR_CUDA, "cow_load_scene: %s", cudaGetErrorString(e)));
    }
    for (size_t i = 0; i < table.size(); i++)
        if (table[i].parent >= 0) c->blocks[(size_t)table[i].parent].children.push_back((int32_t)i);
    c->recs.resize(table.size());
    for (size_t i = 0; i < table.size(); i++) c->recs[i] = block_record(c, c->blocks[i]);
    e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) return bail(fail(COW_ERR_CUDA, "cow_load_scene: %s", cudaGetErrorString(e)));
    *out = c;
    return COW_OK;
}

}  // extern "C"
