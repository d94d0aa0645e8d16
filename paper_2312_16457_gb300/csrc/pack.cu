// pack.cu -- K4 quantize / pack and K5 occupancy build.
//
// K4: FP32 master (8 interleaved channels) -> storage format, after
// multiplying channel c by an exact power of two (the inverse of its scale).
// Conversions round to nearest even; FP8 E4M3 saturates at +-448.
// K5: occupancy bit of a cell = any grid vertex of the cell's closed vertex
// range has ch0 > ln(threshold), compared in double (Sec. 4.5 bakes a binary
// occupancy grid used for empty-space skipping).
#include "cow_common.cuh"
#include "cow_kernels.h"

namespace cow {

namespace {

__global__ void k_amax8(const float *__restrict__ x, int64_t n_vec, unsigned *amax_bits) {
    float m[8] = {0, 0, 0, 0, 0, 0, 0, 0};
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n_vec; i += (int64_t)gridDim.x * blockDim.x) {
        const float4 a = __ldg(reinterpret_cast<const float4 *>(x) + 2 * i);
        const float4 b = __ldg(reinterpret_cast<const float4 *>(x) + 2 * i + 1);
        m[0] = fmaxf(m[0], fabsf(a.x)); m[1] = fmaxf(m[1], fabsf(a.y));
        m[2] = fmaxf(m[2], fabsf(a.z)); m[3] = fmaxf(m[3], fabsf(a.w));
        m[4] = fmaxf(m[4], fabsf(b.x)); m[5] = fmaxf(m[5], fabsf(b.y));
        m[6] = fmaxf(m[6], fabsf(b.z)); m[7] = fmaxf(m[7], fabsf(b.w));
    }
#pragma unroll
    for (int c = 0; c < 8; c++) {
        float v = m[c];
        for (int off = 16; off > 0; off >>= 1) v = fmaxf(v, __shfl_xor_sync(0xffffffffu, v, off));
        // non-negative floats order like their bit patterns
        if ((threadIdx.x & 31) == 0) atomicMax(amax_bits + c, __float_as_uint(v));
    }
}

// Encode one 8-channel vector (already scaled) into its storage bytes.
template <int DT>
__device__ __forceinline__ void encode8(const float v[8], uint32_t w[4]) {
    if (DT == kF16) {
#pragma unroll
        for (int k = 0; k < 4; k++) {
            __half2 h = __floats2half2_rn(v[2 * k], v[2 * k + 1]);
            w[k] = *reinterpret_cast<uint32_t *>(&h);
        }
    } else if (DT == kBF16) {
#pragma unroll
        for (int k = 0; k < 4; k++) {
            __nv_bfloat162 h = __floats2bfloat162_rn(v[2 * k], v[2 * k + 1]);
            w[k] = *reinterpret_cast<uint32_t *>(&h);
        }
    } else if (DT == kFP8) {
#pragma unroll
        for (int k = 0; k < 2; k++) {
            const __nv_fp8x2_storage_t lo =
                __nv_cvt_float2_to_fp8x2(make_float2(v[4 * k], v[4 * k + 1]), __NV_SATFINITE, __NV_E4M3);
            const __nv_fp8x2_storage_t hi =
                __nv_cvt_float2_to_fp8x2(make_float2(v[4 * k + 2], v[4 * k + 3]), __NV_SATFINITE, __NV_E4M3);
            w[k] = (uint32_t)lo | ((uint32_t)hi << 16);
        }
        w[2] = w[3] = 0u;
    }
}

__device__ __forceinline__ void load_scaled(const float *x, int64_t i, const float s[8], float v[8]) {
    const float4 a = __ldg(reinterpret_cast<const float4 *>(x) + 2 * i);
    const float4 b = __ldg(reinterpret_cast<const float4 *>(x) + 2 * i + 1);
    const float r[8] = {a.x, a.y, a.z, a.w, b.x, b.y, b.z, b.w};
#pragma unroll
    for (int c = 0; c < 8; c++) v[c] = __fmul_rn(r[c], s[c]);  // exact: power-of-two factor
}

// FP32: natural layout.  FP16 / BF16 / FP8: pair layout, element i = (vertex
// i, vertex i+1) along rows of `row` vertices (the last of a row repeats).
template <int DT>
__global__ void k_pack(const float *__restrict__ x, int64_t n_vec, int row, const float *__restrict__ inv_scale,
                       void *out) {
    float s[8];
#pragma unroll
    for (int c = 0; c < 8; c++) s[c] = inv_scale[c];
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n_vec; i += (int64_t)gridDim.x * blockDim.x) {
        float v[8];
        load_scaled(x, i, s, v);
        if (DT == kF32) {
            float4 *o = reinterpret_cast<float4 *>(out) + 2 * i;
            o[0] = make_float4(v[0], v[1], v[2], v[3]);
            o[1] = make_float4(v[4], v[5], v[6], v[7]);
            continue;
        }
        const int64_t j = (i % row) == row - 1 ? i : i + 1;
        float vn[8];
        load_scaled(x, j, s, vn);
        uint32_t a[4], b[4];
        encode8<DT>(v, a);
        encode8<DT>(vn, b);
        if (DT == kFP8) {
            reinterpret_cast<uint4 *>(out)[i] = make_uint4(a[0], a[1], b[0], b[1]);
        } else {
            uint4 *o = reinterpret_cast<uint4 *>(out) + 2 * i;
            o[0] = make_uint4(a[0], a[1], a[2], a[3]);
            o[1] = make_uint4(b[0], b[1], b[2], b[3]);
        }
    }
}

__global__ void k_occupancy(const float *__restrict__ grid, int R, int C, int Nc, double lt, uint32_t *bits) {
    const int64_t ncell = (int64_t)Nc * Nc * Nc;
    for (int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; c < ncell; c += (int64_t)gridDim.x * blockDim.x) {
        const int cx = (int)(c % Nc), cy = (int)((c / Nc) % Nc), cz = (int)(c / ((int64_t)Nc * Nc));
        bool on = false;
        const int z1 = min(cz * C + C, R - 1), y1 = min(cy * C + C, R - 1), x1 = min(cx * C + C, R - 1);
        for (int z = cz * C; z <= z1 && !on; z++)
            for (int y = cy * C; y <= y1 && !on; y++)
                for (int x = cx * C; x <= x1; x++)
                    if ((double)__ldg(grid + ((((int64_t)z * R + y) * R + x) << 3)) > lt) {
                        on = true;
                        break;
                    }
        if (on) atomicOr(bits + (c >> 5), 1u << (c & 31));
    }
}

// FP8 quad layout (planes of the mixed format): element (u, v) of a P x P
// plane holds the FP8 texels (u, v), (u+1, v), (u, v+1), (u+1, v+1), clamped
// at the last row and column, 8 bytes each.
__global__ void k_pack_quad8(const float *__restrict__ x, int P, const float *__restrict__ inv_scale, void *out) {
    float s[8];
#pragma unroll
    for (int c = 0; c < 8; c++) s[c] = inv_scale[c];
    const int64_t n = (int64_t)P * P;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const int u = (int)(i % P), v = (int)(i / P);
        const int u1 = min(u + 1, P - 1), v1 = min(v + 1, P - 1);
        const int64_t t[4] = {(int64_t)v * P + u, (int64_t)v * P + u1, (int64_t)v1 * P + u, (int64_t)v1 * P + u1};
        uint32_t w[8];
#pragma unroll
        for (int q = 0; q < 4; q++) {
            float val[8];
            load_scaled(x, t[q], s, val);
            uint32_t e[4];
            encode8<kFP8>(val, e);
            w[2 * q] = e[0];
            w[2 * q + 1] = e[1];
        }
        uint4 *o = reinterpret_cast<uint4 *>(out) + 2 * i;
        o[0] = make_uint4(w[0], w[1], w[2], w[3]);
        o[1] = make_uint4(w[4], w[5], w[6], w[7]);
    }
}

// Grid packing into any layout, dense or brick-sparse.  Output element e is
// the element of the voxel corner (x, y, z):
//   dense        e = (z R + y) R + x (sy = R, sz = R^2);
//   brick-sparse e = s belem + lz sz + ly sy + lx: slot s holds brick
//                blist[s] = (bz Nb + by) Nb + bx and (x, y, z) = kBrick (bx,
//                by, bz) + (lx, ly, lz);
// coordinates beyond R - 1 are clamped (elements never read by a lookup).
// Layouts: kLayNat one vertex (FP32); kLayPair vertices x, x+1; kLayQuad8
// the FP8 vertices (x..x+1, y..y+1) of slice z; kLayOct16 channel 0 of the
// eight corners in BF16 (unscaled), corner k = dx + 2 dy + 4 dz.
__global__ void __launch_bounds__(256) k_pack_grid(const float *__restrict__ x, int R, int64_t n_elem, int sy, int sz,
                                                   int belem, const int32_t *__restrict__ blist, int nb, int dtype,
                                                   int lay, const float *__restrict__ inv_scale, void *out) {
    float s[8];
#pragma unroll
    for (int c = 0; c < 8; c++) s[c] = inv_scale ? inv_scale[c] : 1.0f;
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < n_elem; e += (int64_t)gridDim.x * blockDim.x) {
        int64_t r = e;
        int ox = 0, oy = 0, oz = 0;
        if (blist) {
            const int64_t slot = e / belem;
            r = e - slot * belem;
            const int bid = blist[slot];
            ox = (bid % nb) << kBrickLog2;
            oy = ((bid / nb) % nb) << kBrickLog2;
            oz = (bid / (nb * nb)) << kBrickLog2;
        }
        const int lz = (int)(r / sz), rem = (int)(r - (int64_t)lz * sz);
        const int ly = rem / sy, lx = rem - ly * sy;
        const int vx = min(ox + lx, R - 1), vy = min(oy + ly, R - 1), vz = min(oz + lz, R - 1);
        const int vx1 = min(vx + 1, R - 1), vy1 = min(vy + 1, R - 1), vz1 = min(vz + 1, R - 1);
        auto vid = [&](int xx, int yy, int zz) { return ((int64_t)zz * R + yy) * R + xx; };
        if (lay == kLayOct16) {
            uint32_t w[4];
#pragma unroll
            for (int j = 0; j < 4; j++) {
                const int yy = (j & 1) ? vy1 : vy, zz = (j >> 1) ? vz1 : vz;
                const float a = __ldg(x + 8 * vid(vx, yy, zz)), b2 = __ldg(x + 8 * vid(vx1, yy, zz));
                __nv_bfloat162 h = __floats2bfloat162_rn(a, b2);
                w[j] = *reinterpret_cast<uint32_t *>(&h);
            }
            reinterpret_cast<uint4 *>(out)[e] = make_uint4(w[0], w[1], w[2], w[3]);
        } else if (lay == kLayQuad8) {
            const int64_t t[4] = {vid(vx, vy, vz), vid(vx1, vy, vz), vid(vx, vy1, vz), vid(vx1, vy1, vz)};
            uint32_t w[8];
#pragma unroll
            for (int q = 0; q < 4; q++) {
                float val[8];
                load_scaled(x, t[q], s, val);
                uint32_t enc[4];
                encode8<kFP8>(val, enc);
                w[2 * q] = enc[0];
                w[2 * q + 1] = enc[1];
            }
            uint4 *o = reinterpret_cast<uint4 *>(out) + 2 * e;
            o[0] = make_uint4(w[0], w[1], w[2], w[3]);
            o[1] = make_uint4(w[4], w[5], w[6], w[7]);
        } else if (lay == kLayNat) {
            float v[8];
            load_scaled(x, vid(vx, vy, vz), s, v);
            float4 *o = reinterpret_cast<float4 *>(out) + 2 * e;
            o[0] = make_float4(v[0], v[1], v[2], v[3]);
            o[1] = make_float4(v[4], v[5], v[6], v[7]);
        } else {  // kLayPair
            float v[8], vn[8];
            load_scaled(x, vid(vx, vy, vz), s, v);
            load_scaled(x, vid(vx1, vy, vz), s, vn);
            uint32_t a[4], b2[4];
            if (dtype == kF16) {
                encode8<kF16>(v, a);
                encode8<kF16>(vn, b2);
            } else if (dtype == kBF16) {
                encode8<kBF16>(v, a);
                encode8<kBF16>(vn, b2);
            } else {
                encode8<kFP8>(v, a);
                encode8<kFP8>(vn, b2);
            }
            if (dtype == kFP8) {
                reinterpret_cast<uint4 *>(out)[e] = make_uint4(a[0], a[1], b2[0], b2[1]);
            } else {
                uint4 *o = reinterpret_cast<uint4 *>(out) + 2 * e;
                o[0] = make_uint4(a[0], a[1], a[2], a[3]);
                o[1] = make_uint4(b2[0], b2[1], b2[2], b2[3]);
            }
        }
    }
}

int grid_for(int64_t n, int threads) {
    int64_t b = (n + threads - 1) / threads;
    if (b > 152 * 64) b = 152 * 64;
    return (int)(b < 1 ? 1 : b);
}

}  // namespace

cudaError_t launch_amax8(const float *x, int64_t n_vec, unsigned *amax_bits, cudaStream_t st) {
    cudaError_t e = cudaMemsetAsync(amax_bits, 0, 8 * sizeof(unsigned), st);
    if (e != cudaSuccess) return e;
    k_amax8<<<grid_for(n_vec, 256), 256, 0, st>>>(x, n_vec, amax_bits);
    return cudaGetLastError();
}

cudaError_t launch_pack(const float *x, int64_t n_vec, int row, int dtype, const float *inv_scale8, void *out,
                        cudaStream_t st) {
    const int g = grid_for(n_vec, 256);
    switch (dtype) {
    case kF32: k_pack<kF32><<<g, 256, 0, st>>>(x, n_vec, row, inv_scale8, out); break;
    case kF16: k_pack<kF16><<<g, 256, 0, st>>>(x, n_vec, row, inv_scale8, out); break;
    case kBF16: k_pack<kBF16><<<g, 256, 0, st>>>(x, n_vec, row, inv_scale8, out); break;
    case kFP8: k_pack<kFP8><<<g, 256, 0, st>>>(x, n_vec, row, inv_scale8, out); break;
    default: return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
}

cudaError_t launch_pack_quad8(const float *x, int P, const float *inv_scale8, void *out, cudaStream_t st) {
    k_pack_quad8<<<grid_for((int64_t)P * P, 256), 256, 0, st>>>(x, P, inv_scale8, out);
    return cudaGetLastError();
}

cudaError_t launch_pack_grid(const float *x, int R, int64_t n_elem, int sy, int sz, int belem, const int32_t *blist,
                             int nb, int dtype, int layout, const float *inv_scale8, void *out, cudaStream_t st) {
    if (n_elem <= 0) return cudaSuccess;
    k_pack_grid<<<grid_for(n_elem, 256), 256, 0, st>>>(x, R, n_elem, sy, sz, belem, blist, nb, dtype, layout,
                                                       inv_scale8, out);
    return cudaGetLastError();
}

cudaError_t launch_occupancy(const float *grid, int R, int C, double log_thresh, uint32_t *bits, cudaStream_t st) {
    const int Nc = (R - 1 + C - 1) / C;
    const int64_t ncell = (int64_t)Nc * Nc * Nc;
    cudaError_t e = cudaMemsetAsync(bits, 0, (size_t)((ncell + 31) / 32) * 4, st);
    if (e != cudaSuccess) return e;
    k_occupancy<<<grid_for(ncell, 128), 128, 0, st>>>(grid, R, C, Nc, log_thresh, bits);
    return cudaGetLastError();
}

}  // namespace cow
