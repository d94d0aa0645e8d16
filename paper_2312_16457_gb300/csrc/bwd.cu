// bwd.cu -- K6 / K7: gradients of the rendered colour with respect to every
// grid, plane and deferred-MLP parameter, for the ray-batch form.
//
// Per ray (one thread), given g = dL/dC:
//   K7  recompute the deferred MLP (Eq. 3) from the forward's saved C_d, F and
//       back-propagate it: dL/dC_d = g + dPhi/dC_d^T g, dL/dF, and the ray's
//       contribution to dL/dW (outer products kept in shared memory).
//   K6  re-march the ray over exactly the forward's samples (same sequence
//       code) with the transmittance T and the running prefix sums P_C, P_F;
//       the contribution of the samples after i is the saved total minus the
//       prefix, so no sample is stored.  With e = 1 - alpha = exp(-sigma delta)
//       and the weights of Eq. 1 (w_i = T_i alpha_i):
//         dL/dc_i  = w_i gC,   dL/ds_i = w_i gF
//         dL/dalpha_i = T_i (gC.c_i + gF.s_i) - (gC.S_C + gF.S_F) / e_i
//         dL/df0  = dL/dalpha_i * sigma delta e_i
//                 = sigma delta (T_i e_i (gC.c_i + gF.s_i) - (gC.S_C + gF.S_F))
//       (no division), then dL/df = dL/df0, c(1-c) dL/dc, s(1-s) dL/ds is
//       scattered with the interpolation weights to the 8 grid vertices and
//       12 plane texels (float4 atomics into FP32 gradient arrays in the
//       natural layout).
// The CTA's MLP weight gradient (499 sums over its 128 rays) goes to a
// per-CTA scratch row; a second kernel adds the rows in a fixed order, so the
// MLP gradient does not depend on scheduling.
#include "cow_common.cuh"
#include "cow_kernels.h"
#include "march_core.cuh"

namespace cow {

namespace {

#ifndef COW_BWD_MIN_BLOCKS
// CTAs per SM the re-march's register budget is sized for: 2 lets it keep its
// ~168 live registers (the compiler's own choice, 128, spills); measured on
// the 2x2-block fit: 2 -> 296 ms a step, 3 -> 300, 4 or unset -> 312
#define COW_BWD_MIN_BLOCKS 2
#endif

#ifndef COW_REG_MIN_BLOCKS
// the same for the opacity regulariser's double march: 2 CTAs per SM took a
// regularised fit step from ~496 to ~473 ms
#define COW_REG_MIN_BLOCKS 2
#endif

constexpr int kBwdThreads = kBwdCtaThreads;
constexpr int kVec = 77;  // x (10), dz1 (16), h1 (16), dz2 (16), h2 (16), dz3 (3)

// Vector reduction without a returned value (red, not atom: a float4
// atomicAdd compiles to an atomic that returns the old value through L1, and
// those returns kept the backward's L1 pipe saturated).  16-byte aligned.
__device__ __forceinline__ void red_add4(float *dst, float a, float b, float c, float d) {
    asm volatile("red.global.add.v4.f32 [%0], {%1, %2, %3, %4};" ::"l"(dst), "f"(a), "f"(b), "f"(c), "f"(d)
                 : "memory");
}

__device__ __forceinline__ void red_add1(float *dst, float a) {
    asm volatile("red.global.add.f32 [%0], %1;" ::"l"(dst), "f"(a) : "memory");
}

__device__ __forceinline__ void red_add8(float *dst, float s, const float gf[8]) {
    red_add4(dst, s * gf[0], s * gf[1], s * gf[2], s * gf[3]);
    red_add4(dst + 4, s * gf[4], s * gf[5], s * gf[6], s * gf[7]);
}

// Scatter an 8-channel feature gradient to the taps of the lookup at (p, g).
__device__ __forceinline__ void scatter_taps(const BlockRec &b, float *gg, float *const gp[3], const float p[3],
                                             const float g[3], const float gf[8]) {
    float fr[3];
    int c0[3];
#pragma unroll
    for (int a = 0; a < 3; a++) {
        const int v = min(max(__float2int_rd(g[a]), 0), b.R - 2);
        c0[a] = v;
        fr[a] = fminf(fmaxf(g[a], 0.f), (float)(b.R - 1)) - (float)v;
    }
    const int64_t R = b.R;
    const int64_t base = (c0[2] * R + c0[1]) * R + c0[0];
    const float wx[2] = {1.f - fr[0], fr[0]}, wy[2] = {1.f - fr[1], fr[1]}, wz[2] = {1.f - fr[2], fr[2]};
    if (gg) {
#pragma unroll
        for (int k = 0; k < 8; k++) {
            const int dx = k & 1, dy = (k >> 1) & 1, dz = k >> 2;
            red_add8(gg + 8 * (base + (dz * R + dy) * R + dx), (wy[dy] * wz[dz]) * wx[dx], gf);
        }
    }
    float hf[3];
    int h0[3];
#pragma unroll
    for (int a = 0; a < 3; a++) {
        float h = axis_coord(p[a], b.plo[a], b.kp[a]);
        const int u = min(max(__float2int_rd(h), 0), b.P - 2);
        h = fminf(fmaxf(h, 0.f), (float)(b.P - 1));
        h0[a] = u;
        hf[a] = h - (float)u;
    }
    const int64_t P = b.P;
#pragma unroll
    for (int pl = 0; pl < 3; pl++) {
        if (!gp[pl]) continue;
        const int ua = pl == 2 ? 1 : 0, va = pl == 0 ? 1 : 2;
        const int64_t tb = (int64_t)h0[va] * P + h0[ua];
        const float wu[2] = {1.f - hf[ua], hf[ua]}, wv[2] = {1.f - hf[va], hf[va]};
#pragma unroll
        for (int q = 0; q < 4; q++) {
            const int du = q & 1, dv = q >> 1;
            red_add8(gp[pl] + 8 * (tb + dv * P + du), wv[dv] * wu[du], gf);
        }
    }
}

// K7: deferred-MLP backward per ray; writes (dL/dC_d, dL/dF) of the ray to
// a.gcf (8 floats per ray) and the CTA's 499 weight-gradient sums to its row.
__global__ void __launch_bounds__(kBwdThreads) k_mlp_backward(BwdArgs a) {
    __shared__ float s_w[kMlpParams + 1];
    __shared__ float s_vec[kBwdThreads][kVec];
    for (int i = threadIdx.x; i < kMlpParams; i += blockDim.x) s_w[i] = __ldg(a.mlp + i);
    __syncthreads();
    const int64_t r = (int64_t)blockIdx.x * kBwdThreads + threadIdx.x;
    float *vec = s_vec[threadIdx.x];
    if (r >= a.n_rays) {
        for (int k = 0; k < kVec; k++) vec[k] = 0.f;
    } else {
        const float *w = s_w;
        float x[10], gC[3], gF[4];
#pragma unroll
        for (int c = 0; c < 7; c++) x[c] = __ldg(a.aux + 8 * r + c);
#pragma unroll
        for (int c = 0; c < 3; c++) {
            x[7 + c] = __ldg(a.ray_d + 3 * r + c);
            gC[c] = __ldg(a.dL_drgb + 3 * r + c);
        }
        float dz3[3];
#pragma unroll 1
        for (int j = 0; j < 16; j++) {
            float s = w[kOffB1 + j];
#pragma unroll
            for (int i = 0; i < 10; i++) s = fmaf(x[i], w[kOffW1 + i * 16 + j], s);
            vec[26 + j] = fmaxf(s, 0.f);  // h1
        }
#pragma unroll 1
        for (int j = 0; j < 16; j++) {
            float s = w[kOffB2 + j];
#pragma unroll
            for (int i = 0; i < 16; i++) s = fmaf(vec[26 + i], w[kOffW2 + i * 16 + j], s);
            vec[58 + j] = fmaxf(s, 0.f);  // h2
        }
#pragma unroll
        for (int j = 0; j < 3; j++) {
            float s = w[kOffB3 + j];
#pragma unroll
            for (int i = 0; i < 16; i++) s = fmaf(vec[58 + i], w[kOffW3 + i * 3 + j], s);
            const float sg = 1.f / (1.f + expf(-s));
            dz3[j] = gC[j] * sg * (1.f - sg);
            vec[74 + j] = dz3[j];
        }
#pragma unroll 1
        for (int i = 0; i < 16; i++) {
            float s = 0.f;
#pragma unroll
            for (int j = 0; j < 3; j++) s = fmaf(w[kOffW3 + i * 3 + j], dz3[j], s);
            vec[42 + i] = vec[58 + i] > 0.f ? s : 0.f;  // dz2 (h2 > 0 iff z2 > 0)
        }
#pragma unroll 1
        for (int i = 0; i < 16; i++) {
            float s = 0.f;
#pragma unroll
            for (int j = 0; j < 16; j++) s = fmaf(w[kOffW2 + i * 16 + j], vec[42 + j], s);
            vec[10 + i] = vec[26 + i] > 0.f ? s : 0.f;  // dz1 (h1 > 0 iff z1 > 0)
        }
#pragma unroll 1
        for (int i = 0; i < 7; i++) {
            float s = 0.f;
#pragma unroll
            for (int j = 0; j < 16; j++) s = fmaf(w[kOffW1 + i * 16 + j], vec[10 + j], s);
            if (i < 3) gC[i] += s;
            else gF[i - 3] = s;
        }
#pragma unroll
        for (int k = 0; k < 10; k++) vec[k] = x[k];
        float4 *out = reinterpret_cast<float4 *>(a.gcf + 8 * r);
        out[0] = make_float4(gC[0], gC[1], gC[2], gF[0]);
        out[1] = make_float4(gF[1], gF[2], gF[3], 0.f);
    }
    __syncthreads();
    // MLP weight gradient of this CTA's rays -> its scratch row
    float *row = a.partials + (int64_t)blockIdx.x * kMlpParams;
    for (int t = threadIdx.x; t < kMlpParams; t += blockDim.x) {
        int ia, ib;  // vec offsets of the two factors; ia < 0: bias (single factor)
        if (t < kOffB1) { ia = t / 16; ib = 10 + t % 16; }
        else if (t < kOffW2) { ia = -1; ib = 10 + (t - kOffB1); }
        else if (t < kOffB2) { ia = 26 + (t - kOffW2) / 16; ib = 42 + (t - kOffW2) % 16; }
        else if (t < kOffW3) { ia = -1; ib = 42 + (t - kOffB2); }
        else if (t < kOffB3) { ia = 58 + (t - kOffW3) / 3; ib = 74 + (t - kOffW3) % 3; }
        else { ia = -1; ib = 74 + (t - kOffB3); }
        float s = 0.f;
        for (int q = 0; q < kBwdThreads; q++) s = fmaf(ia >= 0 ? s_vec[q][ia] : 1.f, s_vec[q][ib], s);
        row[t] = s;
    }
}

// K6: re-march and scatter the feature gradients.
template <int DT>
__global__ void __launch_bounds__(kBwdThreads, COW_BWD_MIN_BLOCKS) k_remarch_backward(BwdArgs a,
                                                                                const __grid_constant__ RayRecs rr) {
    const int64_t t = (int64_t)blockIdx.x * kBwdThreads + threadIdx.x;
    if (t >= a.n_rays) return;
    const int64_t r = a.ray_perm ? (int64_t)__ldg(a.ray_perm + t) : t;
    float o[3], d[3], Cf[3], Ff[4], gC[3], gF[4];
#pragma unroll
    for (int c = 0; c < 3; c++) {
        o[c] = __ldg(a.ray_o + 3 * r + c);
        d[c] = __ldg(a.ray_d + 3 * r + c);
        Cf[c] = __ldg(a.aux + 8 * r + c);
        gC[c] = __ldg(a.gcf + 8 * r + c);
    }
#pragma unroll
    for (int c = 0; c < 4; c++) {
        Ff[c] = __ldg(a.aux + 8 * r + 3 + c);
        gF[c] = __ldg(a.gcf + 8 * r + 3 + c);
    }
    int order[kMaxRayIds];
    const int n = sort_blocks_for_ray(rr, o, order);
    float inv_d[3], omax;
    ray_setup(d, o, inv_d, omax);
    float T = 1.f, PC[3] = {0.f, 0.f, 0.f}, PF[4] = {0.f, 0.f, 0.f, 0.f};
    for (int k = 0; k < n; k++) {
        const int id = rr.id[order[k]];
        const BlockRec &b = rr.r[order[k]];
        float *gg = a.grad_grid[id];
        float *const gp[3] = {a.grad_planes[3 * id], a.grad_planes[3 * id + 1], a.grad_planes[3 * id + 2]};
        BrickCache bc;
        const bool more = for_each_sample(b, o, d, inv_d, omax, a.err, [&](const float p[3], const float g[3],
                                                                           float delta) {
            float2 f2[4];
            accumulate_sample<DT>(b, p, g, f2, &bc);
            const float f[8] = {f2[0].x, f2[0].y, f2[1].x, f2[1].y, f2[2].x, f2[2].y, f2[3].x, f2[3].y};
            const float sigma = __expf(f[0]);
            const float e = __expf(-sigma * delta);
            const float wt = T * (1.f - e);
            float c[7];
#pragma unroll
            for (int q = 0; q < 7; q++) c[q] = sigmoidf_fast(f[1 + q]);
            float gdot = 0.f, sdot = 0.f;
#pragma unroll
            for (int q = 0; q < 3; q++) {
                PC[q] = fmaf(wt, c[q], PC[q]);
                gdot = fmaf(gC[q], c[q], gdot);
                sdot = fmaf(gC[q], Cf[q] - PC[q], sdot);
            }
#pragma unroll
            for (int q = 0; q < 4; q++) {
                PF[q] = fmaf(wt, c[3 + q], PF[q]);
                gdot = fmaf(gF[q], c[3 + q], gdot);
                sdot = fmaf(gF[q], Ff[q] - PF[q], sdot);
            }
            float gf[8];
            gf[0] = sigma * delta * (T * e * gdot - sdot);
#pragma unroll
            for (int q = 0; q < 3; q++) gf[1 + q] = wt * gC[q] * c[q] * (1.f - c[q]);
#pragma unroll
            for (int q = 0; q < 4; q++) gf[4 + q] = wt * gF[q] * c[3 + q] * (1.f - c[3 + q]);
            scatter_taps(b, gg, gp, p, g, gf);
            T *= e;
            return !(T < a.ert_eps);
        });
        if (!more) break;
    }
}

// ---------------------------------------------------------------------------
// Training-stage regularisers (Sec. 4.3).
//   Sparsity (Eq. 7): alpha(p) = 1 - exp(-sigma(p) delta_b) at given points,
//     in the block containing p (Eq. 4, first in ids); loss += weight/n alpha,
//     d alpha / d f0 = sigma delta (1 - alpha).
//   Opacity (Eq. 8): per ray and block with occupied samples, alpha^k =
//     1 - prod (1 - alpha_i); loss += weight/n H(clamp(alpha^k)) with H the
//     binary entropy and the clamp to [1e-6, 1 - 1e-6];
//     d alpha^k / d f0_i = sigma_i delta (1 - alpha^k).  The block is marched
//     once for alpha^k -- or alpha^k comes from the forward's in-block
//     transmittance -- and once to scatter.
// Gradients reach the density channel only: 20 scalar atomics per point or
// sample (8 grid vertices, 4 texels of each plane).

__device__ __forceinline__ void scatter_ch0(const BlockRec &b, float *gg, float *const gp[3], const float p[3],
                                            const float g[3], float g0) {
    if (gg) {
        float fr[3];
        int c0[3];
#pragma unroll
        for (int a = 0; a < 3; a++) {
            const int v = min(max(__float2int_rd(g[a]), 0), b.R - 2);
            c0[a] = v;
            fr[a] = fminf(fmaxf(g[a], 0.f), (float)(b.R - 1)) - (float)v;
        }
        const int64_t R = b.R;
        const int64_t base = (c0[2] * R + c0[1]) * R + c0[0];
#pragma unroll
        for (int k = 0; k < 8; k++) {
            const int dx = k & 1, dy = (k >> 1) & 1, dz = k >> 2;
            const float w = (dy ? fr[1] : 1.f - fr[1]) * (dz ? fr[2] : 1.f - fr[2]) * (dx ? fr[0] : 1.f - fr[0]);
            red_add1(gg + 8 * (base + (dz * R + dy) * R + dx), w * g0);
        }
    }
    float hf[3];
    int h0[3];
#pragma unroll
    for (int a = 0; a < 3; a++) {
        float h = axis_coord(p[a], b.plo[a], b.kp[a]);
        const int u = min(max(__float2int_rd(h), 0), b.P - 2);
        h = fminf(fmaxf(h, 0.f), (float)(b.P - 1));
        h0[a] = u;
        hf[a] = h - (float)u;
    }
    const int64_t P = b.P;
#pragma unroll
    for (int pl = 0; pl < 3; pl++) {
        if (!gp[pl]) continue;
        const int ua = pl == 2 ? 1 : 0, va = pl == 0 ? 1 : 2;
        const int64_t tb = (int64_t)h0[va] * P + h0[ua];
#pragma unroll
        for (int q = 0; q < 4; q++) {
            const int du = q & 1, dv = q >> 1;
            const float w = (dv ? hf[va] : 1.f - hf[va]) * (du ? hf[ua] : 1.f - hf[ua]);
            red_add1(gp[pl] + 8 * (tb + dv * P + du), w * g0);
        }
    }
}

// sum of v over the CTA, added to *loss by one thread
__device__ __forceinline__ void add_loss(float v, float *loss) {
    __shared__ float s_part[32];
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) v += __shfl_xor_sync(0xffffffffu, v, off);
    if ((threadIdx.x & 31) == 0) s_part[threadIdx.x >> 5] = v;
    __syncthreads();
    if (threadIdx.x < 32) {
        float w = threadIdx.x < (blockDim.x >> 5) ? s_part[threadIdx.x] : 0.f;
#pragma unroll
        for (int off = 16; off > 0; off >>= 1) w += __shfl_xor_sync(0xffffffffu, w, off);
        if (threadIdx.x == 0 && loss) atomicAdd(loss, w);
    }
}

template <int DT>
__global__ void __launch_bounds__(kBwdThreads) k_sparsity(RegArgs a, const __grid_constant__ RayRecs rr) {
    const int64_t r = (int64_t)blockIdx.x * kBwdThreads + threadIdx.x;
    float term = 0.f;
    if (r < a.n) {
        const float p[3] = {__ldg(a.pts + 3 * r), __ldg(a.pts + 3 * r + 1), __ldg(a.pts + 3 * r + 2)};
        int pos = -1;
        for (int k = 0; k < rr.n && pos < 0; k++) {
            const BlockRec &bc = rr.r[k];
            if ((bc.unb & kUnbContracted) ? owned_unbounded(bc, p) : inside_block(bc, p)) pos = k;
        }
        if (pos >= 0) {
            const int id = rr.id[pos];
            const BlockRec &b = rr.r[pos];
            float q[3], g[3];
            lookup_coords(b, p, q, g);
            float2 f2[4];
            accumulate_sample<DT>(b, q, g, f2);
            const float sigma = expf(f2[0].x);
            const float alpha = -expm1f(-sigma * b.delta);
            const float scale = a.weight / (float)a.n;
            term = scale * alpha;
            if (a.grad_grid) {
                float *const gp[3] = {a.grad_planes[3 * id], a.grad_planes[3 * id + 1], a.grad_planes[3 * id + 2]};
                scatter_ch0(b, a.grad_grid[id], gp, q, g, scale * sigma * b.delta * (1.f - alpha));
            }
        }
    }
    add_loss(term, a.loss);
}

template <int DT>
__global__ void __launch_bounds__(kBwdThreads, COW_REG_MIN_BLOCKS) k_opacity(RegArgs a,
                                                                          const __grid_constant__ RayRecs rr) {
    const int64_t t = (int64_t)blockIdx.x * kBwdThreads + threadIdx.x;
    float term = 0.f;
    if (t < a.n) {
        const int64_t r = a.ray_perm ? (int64_t)__ldg(a.ray_perm + t) : t;
        float o[3], d[3];
#pragma unroll
        for (int c = 0; c < 3; c++) {
            o[c] = __ldg(a.ray_o + 3 * r + c);
            d[c] = __ldg(a.ray_d + 3 * r + c);
        }
        int order[kMaxRayIds];
        const int n = sort_blocks_for_ray(rr, o, order);
        float inv_d[3], omax;
        ray_setup(d, o, inv_d, omax);
        const float scale = a.weight / (float)a.n, eps = 1e-6f;
        for (int k = 0; k < n; k++) {
            const int id = rr.id[order[k]];
            const BlockRec &b = rr.r[order[k]];
            float T = 1.f;
            if (a.block_T) {  // the forward's in-block transmittance
                T = __ldg(a.block_T + r * rr.n + order[k]);
                if (T < 0.f) continue;  // no occupied sample
            } else {
                int nk = 0;
                BrickCache bc;
                for_each_sample(b, o, d, inv_d, omax, a.err, [&](const float p[3], const float g[3], float delta) {
                    float2 f2[4];
                    accumulate_sample<DT>(b, p, g, f2, &bc);
                    T *= expf(-expf(f2[0].x) * delta);
                    nk++;
                    return true;
                });
                if (nk == 0) continue;
            }
            const float a_raw = 1.f - T;
            const float al = fminf(fmaxf(a_raw, eps), 1.f - eps);
            term -= scale * (al * logf(al) + (1.f - al) * log1pf(-al));
            if (!a.grad_grid || !(a_raw > eps && a_raw < 1.f - eps)) continue;
            const float ga = -scale * (logf(al) - log1pf(-al));  // d loss / d alpha^k
            float *gg = a.grad_grid[id];
            float *const gp[3] = {a.grad_planes[3 * id], a.grad_planes[3 * id + 1], a.grad_planes[3 * id + 2]};
            BrickCache bc;
            for_each_sample(b, o, d, inv_d, omax, a.err, [&](const float p[3], const float g[3], float delta) {
                float2 f2[4];
                accumulate_sample<DT>(b, p, g, f2, &bc);
                scatter_ch0(b, gg, gp, p, g, ga * expf(f2[0].x) * delta * T);
                return true;
            });
        }
    }
    add_loss(term, a.loss);
}

// grad_mlp[t] += sum over CTA rows, in row order
__global__ void k_reduce_rows(const float *__restrict__ partials, int n_rows, float *grad_mlp) {
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= kMlpParams) return;
    float s = 0.f;
    for (int k = 0; k < n_rows; k++) s += partials[(int64_t)k * kMlpParams + t];
    grad_mlp[t] += s;
}

__global__ void k_adam(float *__restrict__ p, const float *__restrict__ g, float *__restrict__ m,
                       float *__restrict__ v, int64_t n, float lr, float b1, float b2, float eps, float bc1,
                       float bc2) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const float gi = g[i];
        const float mi = b1 * m[i] + (1.f - b1) * gi;
        const float vi = b2 * v[i] + (1.f - b2) * gi * gi;
        m[i] = mi;
        v[i] = vi;
        p[i] -= lr * (mi / bc1) / (sqrtf(vi / bc2) + eps);
    }
}

__global__ void k_mse_grad(const float *__restrict__ rgb, const float *__restrict__ tgt, int64_t n, float scale,
                           float *__restrict__ grad, float *loss) {
    __shared__ float s_part[32];
    float acc = 0.f;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const float e = rgb[i] - tgt[i];
        grad[i] = 2.f * scale * e;
        acc = fmaf(e, e, acc);
    }
    for (int off = 16; off > 0; off >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, off);
    if ((threadIdx.x & 31) == 0) s_part[threadIdx.x >> 5] = acc;
    __syncthreads();
    if (threadIdx.x < 32) {
        float v = threadIdx.x < (blockDim.x >> 5) ? s_part[threadIdx.x] : 0.f;
        for (int off = 16; off > 0; off >>= 1) v += __shfl_xor_sync(0xffffffffu, v, off);
        if (threadIdx.x == 0 && loss) atomicAdd(loss, v * scale);
    }
}

// ---------------------------------------------------------------------------
// Per-block MLP form (Eq. 5 with Eq. 3 per block):
//   C = sum_k B_k X_k,  X_k = C^k + Phi^k(C^k, F^k, PE(d)),  B_{k+1} = B_k (1 - alpha^k)
// over the blocks with occupied samples.  Three passes, ray by ray:
//   P1  march every block once: C^k, F^k and B_k to scratch S;
//   P2  per (ray, block): Phi^k backward with u = B_k dL/dC gives
//       dL/dC^k = u + J_C^T u, dL/dF^k = J_F^T u and dL/dC . X_k (scratch G),
//       and adds u's weight gradient to block k's MLP gradient;
//   P3  march every block again and scatter the feature gradients: with
//       Q_k = sum_{j>k} B_j dL/dC . X_j (the later blocks' dependence on
//       1 - alpha^k), the Eq. 11 backward of the global form gives
//         dL/df0 = sigma delta (T_i e_i (gC.c_i + gF.s_i) - (gC.S_C + gF.S_F) - Q_k)
//       with in-block T_i and the block's own totals and upstreams.
// No early termination (the ray form's training calls use none).

// The per-block MLP input i: C^k (3), F^k (4), d (3), then sin / cos(2^l d).
__device__ __forceinline__ float bm_input(int i, const float ck[7], const float d[3]) {
    if (i < 7) return ck[i];
    if (i < 10) return d[i - 7];
    const int j = i - 10, l = j / 6, q = j % 6;
    const float v = ldexpf(d[q % 3], l);
    return q < 3 ? sinf(v) : cosf(v);
}

// P1
template <int DT>
__global__ void __launch_bounds__(kBwdThreads) k_bm_pass1(BmBwdArgs a, const __grid_constant__ RayRecs rr) {
    const int64_t t = (int64_t)blockIdx.x * kBwdThreads + threadIdx.x;
    if (t >= a.n_rays) return;
    const int64_t r = a.ray_perm ? (int64_t)__ldg(a.ray_perm + t) : t;
    float o[3], d[3];
#pragma unroll
    for (int c = 0; c < 3; c++) {
        o[c] = __ldg(a.ray_o + 3 * r + c);
        d[c] = __ldg(a.ray_d + 3 * r + c);
    }
    int order[kMaxRayIds];
    const int n = sort_blocks_for_ray(rr, o, order);
    float inv_d[3], omax;
    ray_setup(d, o, inv_d, omax);
    float B = 1.f;
    for (int k = 0; k < n; k++) {
        RayState sb = {{0.f, 0.f, 0.f}, {0.f, 0.f, 0.f, 0.f}, 1.f, 0, false};
        march_block<DT>(rr.r[order[k]], o, d, inv_d, omax, 0.f, sb, a.err);
        float4 *e = reinterpret_cast<float4 *>(a.S + 8 * (r * a.n_ids + order[k]));
        if (sb.nsamp == 0) {
            e[1] = make_float4(0.f, 0.f, 0.f, -1.f);
            continue;
        }
        e[0] = make_float4(sb.Cd[0], sb.Cd[1], sb.Cd[2], sb.F[0]);
        e[1] = make_float4(sb.F[1], sb.F[2], sb.F[3], B);
        B *= sb.T;
    }
}

// A weight-gradient term summed over the warp's 32 rays, then one reduction.
__device__ __forceinline__ void warp_red(float *dst, float v) {
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) v += __shfl_xor_sync(0xffffffffu, v, off);
    if ((threadIdx.x & 31) == 0) red_add1(dst, v);
}

// Sixteen weight-gradient terms (dst[0 .. 15]) summed over the warp's 32 rays
// at once: the two half-warps are folded, then at each of the four remaining
// lane bits every lane keeps one half of its values and adds the partner's
// copy of that half, so lane l ends with the warp sum of term l & 15 -- 31
// shuffles for the sixteen sums instead of 80 -- and lanes 0-15 reduce one
// term each.  v is overwritten.
__device__ __forceinline__ void warp_red16(float *dst, float v[16]) {
    const int lane = threadIdx.x & 31;
#pragma unroll
    for (int j = 0; j < 16; j++) v[j] += __shfl_xor_sync(0xffffffffu, v[j], 16);
#pragma unroll
    for (int s = 8; s >= 1; s >>= 1) {
        const bool up = (lane & s) != 0;
#pragma unroll
        for (int j = 0; j < s; j++) {
            const float send = up ? v[j] : v[j + s];
            const float keep = up ? v[j + s] : v[j];
            v[j] = keep + __shfl_xor_sync(0xffffffffu, send, s);
        }
    }
    if (lane < 16) red_add1(dst + lane, v[0]);
}

// P2: one thread per (ray, block) pair.  The pairs are laid out block-major
// with each block's rays padded to a multiple of 32, so a warp holds one
// block for 32 rays and sums that block's weight gradients before reducing;
// padding lanes and blocks a ray has no sample in take part with zeros.
__global__ void __launch_bounds__(kBwdThreads) k_bm_mlp(BmBwdArgs a, const __grid_constant__ RayRecs rr) {
    const int64_t t = (int64_t)blockIdx.x * kBwdThreads + threadIdx.x;
    const int64_t rows = (a.n_rays + 31) & ~(int64_t)31;
    const int k = (int)min(t / rows, (int64_t)a.n_ids - 1);  // warp-uniform
    const int64_t r = t - (int64_t)k * rows;
    const bool ray = t < rows * a.n_ids && r < a.n_rays;
    const int64_t pe = r * a.n_ids + k;  // the pair's scratch entry
    float4 e0 = make_float4(0.f, 0.f, 0.f, 0.f), e1 = make_float4(0.f, 0.f, 0.f, -1.f);
    if (ray) {
        const float4 *e = reinterpret_cast<const float4 *>(a.S + 8 * pe);
        e0 = e[0];
        e1 = e[1];
    }
    const bool act = ray && e1.w >= 0.f;
    if (!act) {  // the scratch of a block without samples holds no C^k, F^k: zeros, not stale values
        e0 = make_float4(0.f, 0.f, 0.f, 0.f);
        e1 = make_float4(0.f, 0.f, 0.f, 0.f);
    }
    const float ck[7] = {e0.x, e0.y, e0.z, e0.w, e1.x, e1.y, e1.z};
    const float B = act ? e1.w : 0.f;
    float d[3], g[3], u[3];
#pragma unroll
    for (int c = 0; c < 3; c++) {
        d[c] = ray ? __ldg(a.ray_d + 3 * r + c) : 0.f;
        g[c] = ray ? __ldg(a.dL_drgb + 3 * r + c) : 0.f;
        u[c] = B * g[c];
    }
    const int id = rr.id[k];
    const int n_in = 10 + 6 * a.n_freq;
    const float *W1 = a.mlps + (int64_t)id * a.mlp_stride;
    const float *b1 = W1 + n_in * 16, *W2 = b1 + 16, *b2 = W2 + 256, *W3 = b2 + 16, *b3 = W3 + 48;
    float *gW1 = a.grad_mlps + (int64_t)id * a.grad_stride;
    float *gb1 = gW1 + n_in * 16, *gW2 = gb1 + 16, *gb2 = gW2 + 256, *gW3 = gb2 + 16, *gb3 = gW3 + 48;
    float h1[16], h2[16];
#pragma unroll
    for (int j = 0; j < 16; j++) h1[j] = __ldg(b1 + j);
    for (int i = 0; i < n_in; i++) {
        const float xi = bm_input(i, ck, d);
#pragma unroll
        for (int j = 0; j < 16; j++) h1[j] = fmaf(xi, __ldg(W1 + i * 16 + j), h1[j]);
    }
#pragma unroll
    for (int j = 0; j < 16; j++) h1[j] = fmaxf(h1[j], 0.f);  // h1 > 0 iff z1 > 0
#pragma unroll
    for (int j = 0; j < 16; j++) {
        float z = __ldg(b2 + j);
#pragma unroll
        for (int i = 0; i < 16; i++) z = fmaf(h1[i], __ldg(W2 + i * 16 + j), z);
        h2[j] = fmaxf(z, 0.f);
    }
    float phi[3], dz3[3];
#pragma unroll
    for (int j = 0; j < 3; j++) {
        float z = __ldg(b3 + j);
#pragma unroll
        for (int i = 0; i < 16; i++) z = fmaf(h2[i], __ldg(W3 + i * 3 + j), z);
        phi[j] = 1.f / (1.f + expf(-z));
        dz3[j] = u[j] * phi[j] * (1.f - phi[j]);
        warp_red(gb3 + j, dz3[j]);
    }
    float dz2[16];
#pragma unroll
    for (int i = 0; i < 16; i++) {
        float s = 0.f;
#pragma unroll
        for (int j = 0; j < 3; j++) {
            s = fmaf(__ldg(W3 + i * 3 + j), dz3[j], s);
            warp_red(gW3 + i * 3 + j, h2[i] * dz3[j]);
        }
        dz2[i] = h2[i] > 0.f ? s : 0.f;
    }
    float dz1[16], gv[16];
#pragma unroll
    for (int j = 0; j < 16; j++) gv[j] = dz2[j];
    warp_red16(gb2, gv);
#pragma unroll
    for (int i = 0; i < 16; i++) {
        float s = 0.f;
#pragma unroll
        for (int j = 0; j < 16; j++) {
            s = fmaf(__ldg(W2 + i * 16 + j), dz2[j], s);
            gv[j] = h1[i] * dz2[j];
        }
        warp_red16(gW2 + i * 16, gv);
        dz1[i] = h1[i] > 0.f ? s : 0.f;
    }
#pragma unroll
    for (int j = 0; j < 16; j++) gv[j] = dz1[j];
    warp_red16(gb1, gv);
    float gx[7];
    for (int i = 0; i < n_in; i++) {
        const float xi = bm_input(i, ck, d);
        float s = 0.f;
#pragma unroll
        for (int j = 0; j < 16; j++) {
            s = fmaf(__ldg(W1 + i * 16 + j), dz1[j], s);
            gv[j] = xi * dz1[j];
        }
        warp_red16(gW1 + i * 16, gv);
        if (i < 7) gx[i] = s;
    }
    if (!ray) return;
    float4 *go = reinterpret_cast<float4 *>(a.G + 8 * pe);
    if (!act) {
        go[0] = make_float4(0.f, 0.f, 0.f, 0.f);
        go[1] = make_float4(0.f, 0.f, 0.f, 0.f);
        return;
    }
    float xg = 0.f;
#pragma unroll
    for (int c = 0; c < 3; c++) xg = fmaf(g[c], ck[c] + phi[c], xg);
    go[0] = make_float4(u[0] + gx[0], u[1] + gx[1], u[2] + gx[2], gx[3]);
    go[1] = make_float4(gx[4], gx[5], gx[6], xg);
}

// P3
template <int DT>
__global__ void __launch_bounds__(kBwdThreads, COW_BWD_MIN_BLOCKS) k_bm_remarch(BmBwdArgs a,
                                                                          const __grid_constant__ RayRecs rr) {
    const int64_t t = (int64_t)blockIdx.x * kBwdThreads + threadIdx.x;
    if (t >= a.n_rays) return;
    const int64_t r = a.ray_perm ? (int64_t)__ldg(a.ray_perm + t) : t;
    float o[3], d[3];
#pragma unroll
    for (int c = 0; c < 3; c++) {
        o[c] = __ldg(a.ray_o + 3 * r + c);
        d[c] = __ldg(a.ray_d + 3 * r + c);
    }
    const float *S = a.S + 8 * r * a.n_ids, *G = a.G + 8 * r * a.n_ids;
    float Qtot = 0.f;  // sum_k B_k dL/dC . X_k
    for (int k = 0; k < a.n_ids; k++) {
        const float B = __ldg(S + 8 * k + 7);
        if (B >= 0.f) Qtot = fmaf(B, __ldg(G + 8 * k + 7), Qtot);
    }
    int order[kMaxRayIds];
    const int n = sort_blocks_for_ray(rr, o, order);
    float inv_d[3], omax;
    ray_setup(d, o, inv_d, omax);
    float P = 0.f;
    for (int k = 0; k < n; k++) {
        const int idx = order[k];
        const float B = __ldg(S + 8 * idx + 7);
        if (B < 0.f) continue;  // no occupied sample: no part in Eq. 5
        float Cf[3], Ff[4], gC[3], gF[4];
#pragma unroll
        for (int c = 0; c < 3; c++) {
            Cf[c] = __ldg(S + 8 * idx + c);
            gC[c] = __ldg(G + 8 * idx + c);
        }
#pragma unroll
        for (int c = 0; c < 4; c++) {
            Ff[c] = __ldg(S + 8 * idx + 3 + c);
            gF[c] = __ldg(G + 8 * idx + 3 + c);
        }
        P = fmaf(B, __ldg(G + 8 * idx + 7), P);
        const float Q = Qtot - P;  // the blocks behind this one
        const int id = rr.id[idx];
        const BlockRec &b = rr.r[idx];
        float *gg = a.grad_grid[id];
        float *const gp[3] = {a.grad_planes[3 * id], a.grad_planes[3 * id + 1], a.grad_planes[3 * id + 2]};
        float T = 1.f, PC[3] = {0.f, 0.f, 0.f}, PF[4] = {0.f, 0.f, 0.f, 0.f};
        BrickCache bc;
        for_each_sample(b, o, d, inv_d, omax, a.err, [&](const float p[3], const float g[3], float delta) {
            float2 f2[4];
            accumulate_sample<DT>(b, p, g, f2, &bc);
            const float f[8] = {f2[0].x, f2[0].y, f2[1].x, f2[1].y, f2[2].x, f2[2].y, f2[3].x, f2[3].y};
            const float sigma = __expf(f[0]);
            const float e = __expf(-sigma * delta);
            const float wt = T * (1.f - e);
            float c[7];
#pragma unroll
            for (int q = 0; q < 7; q++) c[q] = sigmoidf_fast(f[1 + q]);
            float gdot = 0.f, sdot = Q;
#pragma unroll
            for (int q = 0; q < 3; q++) {
                PC[q] = fmaf(wt, c[q], PC[q]);
                gdot = fmaf(gC[q], c[q], gdot);
                sdot = fmaf(gC[q], Cf[q] - PC[q], sdot);
            }
#pragma unroll
            for (int q = 0; q < 4; q++) {
                PF[q] = fmaf(wt, c[3 + q], PF[q]);
                gdot = fmaf(gF[q], c[3 + q], gdot);
                sdot = fmaf(gF[q], Ff[q] - PF[q], sdot);
            }
            float gf[8];
            gf[0] = sigma * delta * (T * e * gdot - sdot);
#pragma unroll
            for (int q = 0; q < 3; q++) gf[1 + q] = wt * gC[q] * c[q] * (1.f - c[q]);
#pragma unroll
            for (int q = 0; q < 4; q++) gf[4 + q] = wt * gF[q] * c[3 + q] * (1.f - c[3 + q]);
            scatter_taps(b, gg, gp, p, g, gf);
            T *= e;
            return true;
        });
    }
}

}  // namespace

int backward_rows(int64_t n_rays) { return (int)((n_rays + kBwdThreads - 1) / kBwdThreads); }

cudaError_t launch_backward_rays(const BwdArgs &a, const RayRecs &rr, cudaStream_t st) {
    if (a.n_rays <= 0) return cudaSuccess;
    const int nb = backward_rows(a.n_rays);
    k_mlp_backward<<<nb, kBwdThreads, 0, st>>>(a);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    k_reduce_rows<<<(kMlpParams + 127) / 128, 128, 0, st>>>(a.partials, nb, a.grad_mlp);
    {
        const cudaError_t e_ = dispatch_dt(a.dtype, [&](auto D) {
            k_remarch_backward<decltype(D)::value><<<nb, kBwdThreads, 0, st>>>(a, rr);
            return cudaSuccess;
        });
        if (e_ != cudaSuccess) return e_;
    }
    return cudaGetLastError();
}

cudaError_t launch_backward_block_mlps(const BmBwdArgs &a, const RayRecs &rr, cudaStream_t st) {
    if (a.n_rays <= 0) return cudaSuccess;
    const int nb = backward_rows(a.n_rays);
    const int64_t padded = ((a.n_rays + 31) & ~(int64_t)31) * a.n_ids;  // k_bm_mlp's threads
    if (!a.have_state) {
        const cudaError_t e_ = dispatch_dt(a.dtype, [&](auto D) {
            k_bm_pass1<decltype(D)::value><<<nb, kBwdThreads, 0, st>>>(a, rr);
            return cudaSuccess;
        });
        if (e_ != cudaSuccess) return e_;
    }
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    k_bm_mlp<<<(unsigned)((padded + kBwdThreads - 1) / kBwdThreads), kBwdThreads, 0, st>>>(a, rr);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    {
        const cudaError_t e_ = dispatch_dt(a.dtype, [&](auto D) {
            k_bm_remarch<decltype(D)::value><<<nb, kBwdThreads, 0, st>>>(a, rr);
            return cudaSuccess;
        });
        if (e_ != cudaSuccess) return e_;
    }
    return cudaGetLastError();
}

cudaError_t launch_sparsity(const RegArgs &a, const RayRecs &rr, cudaStream_t st) {
    if (a.n <= 0) return cudaSuccess;
    const int nb = (int)((a.n + kBwdThreads - 1) / kBwdThreads);
    {
        const cudaError_t e_ = dispatch_dt(a.dtype, [&](auto D) {
            k_sparsity<decltype(D)::value><<<nb, kBwdThreads, 0, st>>>(a, rr);
            return cudaSuccess;
        });
        if (e_ != cudaSuccess) return e_;
    }
    return cudaGetLastError();
}

cudaError_t launch_opacity(const RegArgs &a, const RayRecs &rr, cudaStream_t st) {
    if (a.n <= 0) return cudaSuccess;
    const int nb = (int)((a.n + kBwdThreads - 1) / kBwdThreads);
    {
        const cudaError_t e_ = dispatch_dt(a.dtype, [&](auto D) {
            k_opacity<decltype(D)::value><<<nb, kBwdThreads, 0, st>>>(a, rr);
            return cudaSuccess;
        });
        if (e_ != cudaSuccess) return e_;
    }
    return cudaGetLastError();
}

cudaError_t launch_adam(float *p, const float *g, float *m, float *v, int64_t n, float lr, float b1, float b2,
                        float eps, int step, cudaStream_t st) {
    if (n <= 0) return cudaSuccess;
    const float bc1 = 1.f - powf(b1, (float)step), bc2 = 1.f - powf(b2, (float)step);
    int64_t blocks = (n + 255) / 256;
    if (blocks > 152 * 32) blocks = 152 * 32;
    k_adam<<<(int)blocks, 256, 0, st>>>(p, g, m, v, n, lr, b1, b2, eps, bc1, bc2);
    return cudaGetLastError();
}

cudaError_t launch_mse_grad(const float *rgb, const float *tgt, int64_t n, float *grad, float *loss, cudaStream_t st) {
    if (n <= 0) return cudaSuccess;
    if (loss) {
        cudaError_t e = cudaMemsetAsync(loss, 0, sizeof(float), st);
        if (e != cudaSuccess) return e;
    }
    int64_t blocks = (n + 255) / 256;
    if (blocks > 152 * 16) blocks = 152 * 16;
    k_mse_grad<<<(int)blocks, 256, 0, st>>>(rgb, tgt, n, 1.0f / (float)n, grad, loss);
    return cudaGetLastError();
}

}  // namespace cow
