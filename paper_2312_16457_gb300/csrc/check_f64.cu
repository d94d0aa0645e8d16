// check_f64.cu -- an FP64 render of ray batches on the GPU, for
// finite-difference checks of the gradient: the same samples as the FP32
// marcher (the FP32 decision sequence of march_core.cuh picks them), then
// every lookup, activation, weight, composite and the deferred MLP in FP64
// from FP64 copies of the features.  A central difference of this render
// is accurate to ~1e-10 relative, so it can check the FP32 backward at the
// differentiation form's 1e-3 tolerance entry by entry.
#include "cow_common.cuh"
#include "cow_kernels.h"
#include "march_core.cuh"

namespace cow {

namespace {

constexpr int kF64Threads = 128;

// Vertex-aligned coordinate of x on an axis of n vertices spanning [lo, hi],
// clamped; the corner and the fraction.
__device__ __forceinline__ void axis64(double x, double lo, double hi, int n, int &c0, double &fr) {
    double g = (x - lo) * (double)(n - 1) / (hi - lo);
    g = fmin(fmax(g, 0.0), (double)(n - 1));
    int c = (int)floor(g);
    c = min(c, n - 2);
    c0 = c;
    fr = g - (double)c;
}

// f = trilinear(grid) + bilinear(xy, xz, yz) at the lookup point q (the
// sample point, or its contraction for an unbounded block), all in FP64.
__device__ void feature64(const BlockRec &b, const double *grid, const double *const planes[3], const float q[3],
                          double f[8]) {
    const bool unb = (b.unb & kUnbContracted) != 0;
    double lo[3], hi[3];
    for (int a = 0; a < 3; a++) {
        lo[a] = unb ? -2.0 : (double)b.lo[a];
        hi[a] = unb ? 2.0 : (double)b.hi[a];
    }
    int c[3];
    double fr[3];
    for (int a = 0; a < 3; a++) axis64((double)q[a], lo[a], hi[a], b.R, c[a], fr[a]);
    for (int k = 0; k < 8; k++) f[k] = 0.0;
    const int64_t R = b.R;
    for (int k = 0; k < 8; k++) {
        const int dx = k & 1, dy = (k >> 1) & 1, dz = k >> 2;
        const double w = (dx ? fr[0] : 1.0 - fr[0]) * (dy ? fr[1] : 1.0 - fr[1]) * (dz ? fr[2] : 1.0 - fr[2]);
        const double *v = grid + 8 * (((c[2] + dz) * R + (c[1] + dy)) * R + (c[0] + dx));
        for (int ch = 0; ch < 8; ch++) f[ch] += w * v[ch];
    }
    int h[3];
    double hf[3];
    for (int a = 0; a < 3; a++) axis64((double)q[a], lo[a], hi[a], b.P, h[a], hf[a]);
    const int64_t P = b.P;
    for (int pl = 0; pl < 3; pl++) {
        const int ua = pl == 2 ? 1 : 0, va = pl == 0 ? 1 : 2;
        for (int k = 0; k < 4; k++) {
            const int du = k & 1, dv = k >> 1;
            const double w = (du ? hf[ua] : 1.0 - hf[ua]) * (dv ? hf[va] : 1.0 - hf[va]);
            const double *v = planes[pl] + 8 * ((h[va] + dv) * P + (h[ua] + du));
            for (int ch = 0; ch < 8; ch++) f[ch] += w * v[ch];
        }
    }
}

__device__ __forceinline__ double sigmoid64(double x) { return 1.0 / (1.0 + exp(-x)); }

__global__ void __launch_bounds__(kF64Threads) k_march_rays_f64(F64Args a, const __grid_constant__ RayRecs rr) {
    const int64_t r = (int64_t)blockIdx.x * kF64Threads + threadIdx.x;
    if (r >= a.n_rays) return;
    float o[3], d[3];
    for (int c = 0; c < 3; c++) {
        o[c] = a.ray_o[3 * r + c];
        d[c] = a.ray_d[3 * r + c];
    }
    int order[kMaxRayIds];
    const int n = sort_blocks_for_ray(rr, o, order);
    float inv_d[3], omax;
    ray_setup(d, o, inv_d, omax);
    double T = 1.0, Cd[3] = {0.0, 0.0, 0.0}, F[4] = {0.0, 0.0, 0.0, 0.0};
    for (int k = 0; k < n; k++) {
        const BlockRec &b = rr.r[order[k]];
        const int id = rr.id[order[k]];
        const double *grid = a.grids[id];
        const double *const planes[3] = {a.planes[3 * id], a.planes[3 * id + 1], a.planes[3 * id + 2]};
        for_each_sample(b, o, d, inv_d, omax, a.err, [&](const float q[3], const float *, float step) {
            double f[8];
            feature64(b, grid, planes, q, f);
            const double sigma = exp(f[0]);
            const double alpha = -expm1(-sigma * (double)step);
            const double w = T * alpha;
            for (int c = 0; c < 3; c++) Cd[c] += w * sigmoid64(f[1 + c]);
            for (int c = 0; c < 4; c++) F[c] += w * sigmoid64(f[4 + c]);
            T *= 1.0 - alpha;
            return true;
        });
    }
    // deferred MLP (Eq. 3), weights input-major as the FP32 path
    const double *m = a.mlp;
    const double x[10] = {Cd[0], Cd[1], Cd[2], F[0], F[1], F[2], F[3], (double)d[0], (double)d[1], (double)d[2]};
    double h1[16], h2[16];
    for (int j = 0; j < 16; j++) {
        double s = m[kOffB1 + j];
        for (int i = 0; i < 10; i++) s += x[i] * m[kOffW1 + i * 16 + j];
        h1[j] = fmax(s, 0.0);
    }
    for (int j = 0; j < 16; j++) {
        double s = m[kOffB2 + j];
        for (int i = 0; i < 16; i++) s += h1[i] * m[kOffW2 + i * 16 + j];
        h2[j] = fmax(s, 0.0);
    }
    for (int j = 0; j < 3; j++) {
        double s = m[kOffB3 + j];
        for (int i = 0; i < 16; i++) s += h2[i] * m[kOffW3 + i * 3 + j];
        a.out_rgb[3 * r + j] = Cd[j] + sigmoid64(s);
    }
    if (a.out_aux) {
        double *ax = a.out_aux + 8 * r;
        for (int c = 0; c < 3; c++) ax[c] = Cd[c];
        for (int c = 0; c < 4; c++) ax[3 + c] = F[c];
        ax[7] = T;
    }
}

}  // namespace

cudaError_t launch_march_rays_f64(const F64Args &a, const RayRecs &rr, cudaStream_t st) {
    if (a.n_rays <= 0) return cudaSuccess;
    const int64_t nb = (a.n_rays + kF64Threads - 1) / kF64Threads;
    k_march_rays_f64<<<(unsigned)nb, kF64Threads, 0, st>>>(a, rr);
    return cudaGetLastError();
}

}  // namespace cow
