/*
 * cow_oracle.c -- plain FP64 CPU oracle for block-based volume rendering of
 * baked MERF-style scene blocks (City-on-Web, arXiv 2312.16457).
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product path may link, load or
 * call this file; only the tests, the package's smoke check and the timed
 * CPU baseline of the benchmark do.  It shares no code, header, table or
 * constant generator with the CUDA library.
 *
 * What it computes (per pixel / per ray), section by section of the paper:
 *   - ray r(t) = o + t d (Sec. 3), pinhole camera, pixel centres;
 *   - ground-plane block partition (Sec. 4.1, Eq. 4): every sample point
 *     belongs to exactly one block, decided with half-open xy boxes;
 *   - baked block feature lookup f^{k,l} (Sec. 4.1 rendering stage, Sec. 4.5):
 *     trilinear sample of a low-resolution 3D grid plus bilinear samples of
 *     three high-resolution planes, summed over 8 channels;
 *   - occupancy grid used to skip samples (Sec. 4.1, Sec. 4.5);
 *   - per-sample opacity alpha = 1 - exp(-sigma delta) and weights (Eq. 1),
 *     diffuse colour and specular feature accumulation (Eq. 2), done per
 *     block as in Eq. 11 of Appendix A;
 *   - cross-block composite in block order (Eq. 5 / Eq. 12), with the
 *     single-pass form (Eq. 14) and the alpha/sum(alpha) blending of the
 *     ablation (Table 4, "no alpha blending") as comparison modes;
 *   - one deferred MLP on the composited features (Eq. 3), or per-block
 *     deferred MLPs with a multi-frequency PE(d) blended by Eq. 5;
 *   - LOD selection, visibility and depth sorting of the real-time viewer
 *     (Appendix D);
 *   - the analytic gradient of the rendered colour with respect to grid,
 *     plane and MLP parameters (reverse mode through the steps above);
 *   - the sparsity (Eq. 7) and block-opacity (Eq. 8) regularisers of
 *     Sec. 4.3 with their gradients.
 *
 * Precision: every continuous quantity (interpolation, activations,
 * compositing, MLP, gradients) is FP64.  The discrete decisions -- which
 * lattice samples exist, which block a sample belongs to, which occupancy
 * cell it falls in, the per-ray block order of the ray-batch form -- are
 * taken on FP32 values computed with one fixed sequence of IEEE-754
 * round-to-nearest operations, so that a GPU that evaluates the same
 * sequence takes bit-identical decisions.  The sample points themselves are
 * those FP32 lattice points.  This file must be compiled with
 * -ffp-contract=off (no fused multiply-add) and without -ffast-math.
 *
 * Parity pins (tests/test_oracle_*.py): closed-form transmittance of a
 * constant-density block, exact reproduction of affine fields, the
 * block-sequential == single-pass equivalence of Appendix A, the failing
 * alpha/sum(alpha) negative control, weight invariants, library float64 MLP,
 * hand-built LOD cases, brute-force occupancy, format definitions of
 * FP16/BF16/FP8-E4M3 and central finite differences for the gradient.
 */
#include <float.h>
#include <math.h>
#include <omp.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#if !defined(FLT_EVAL_METHOD) || FLT_EVAL_METHOD != 0
#error "the FP32 decision sequence needs FLT_EVAL_METHOD == 0"
#endif

#define NCH 8          /* channels: 0 log-density, 1-3 diffuse, 4-7 specular */
#define MLP_IN 10
#define MLP_HID 16
#define MLP_OUT 3
#define MLP_NPARAM 499 /* 10*16+16 + 16*16+16 + 16*3+3 */
#define OFF_W1 0
#define OFF_B1 160
#define OFF_W2 176
#define OFF_B2 432
#define OFF_W3 448
#define OFF_B3 496

typedef struct orc_block {
    float lo[3];
    float hi[3];
    int32_t R;        /* grid vertices per axis */
    int32_t P;        /* plane texels per axis */
    int32_t occ_cell; /* voxels per occupancy-cell edge */
    int32_t level;    /* LOD level, 1 = finest */
    int32_t parent;   /* index of the covering block one level up, -1 if none */
    int32_t is_f64;   /* 1: grid / planes hold double, 0: float */
    const void *grid;       /* R^3 x 8, index ((z*R + y)*R + x)*8 + c */
    const void *planes[3];  /* P^2 x 8 each, index (v*P + u)*8 + c; xy, xz, yz */
    const uint32_t *occ;    /* occupancy bits, NULL = every cell occupied */
    int32_t unbounded;      /* 0, or ORC_CONTRACTED | the xy sides that extend to infinity */
} orc_block;

/* Unbounded boundary blocks (MERF scene contraction, Eq. 16). */
#define ORC_EXT_XLO 1
#define ORC_EXT_XHI 2
#define ORC_EXT_YLO 4
#define ORC_EXT_YHI 8
#define ORC_CONTRACTED 16
#define ORC_CONTRACT_MAX 1.0e4f   /* the march stops beyond ||x||_inf = 1e4 */
#define ORC_CONTRACT_STEPS 65536  /* and after this many steps */

typedef struct orc_camera {
    double c2w[12];   /* 3x4 row-major camera-to-world, OpenGL axes */
    int32_t width, height;
    double fov_y_deg; /* vertical field of view */
} orc_camera;

/* ------------------------------------------------------------------------- */
/* Numeric storage formats, written from their definitions (IEEE-754 binary16,
 * bfloat16 = upper half of binary32, OCP FP8 E4M3 "fn": bias 7, no infinity,
 * max finite 448).  Round to nearest, ties to even.                           */

/* Round |x| to a binary format with `mant` fraction bits and minimum normal
 * exponent `emin`; exact in double because every step is a power-of-two
 * scaling or an integer rounding. */
static double round_to_format(double ax, int mant, int emin) {
    if (ax == 0.0) return 0.0;
    int e;
    frexp(ax, &e);           /* ax = m * 2^e, m in [0.5, 1) */
    e -= 1;                  /* ax = m' * 2^e, m' in [1, 2) */
    if (e < emin) e = emin;  /* subnormal range shares the minimum quantum */
    double q = ldexp(1.0, e - mant);
    return nearbyint(ax / q) * q;   /* default rounding mode: ties to even */
}

uint16_t orc_f32_to_f16(float x) {
    uint32_t bits;
    memcpy(&bits, &x, 4);
    uint16_t sign = (uint16_t)((bits >> 16) & 0x8000u);
    double ax = fabs((double)x);
    if (isnan(x)) return (uint16_t)(sign | 0x7e00u);
    double v = round_to_format(ax, 10, -14);
    if (v >= 65536.0 || isinf(x)) return (uint16_t)(sign | 0x7c00u);
    if (v == 0.0) return sign;
    if (v < ldexp(1.0, -14)) return (uint16_t)(sign | (uint16_t)(v / ldexp(1.0, -24)));
    int e;
    frexp(v, &e);
    e -= 1;
    uint16_t m = (uint16_t)(v / ldexp(1.0, e - 10) - 1024.0);
    return (uint16_t)(sign | (uint16_t)((e + 15) << 10) | m);
}

double orc_f16_to_f64(uint16_t h) {
    int s = (h >> 15) & 1, e = (h >> 10) & 31, m = h & 1023;
    double v;
    if (e == 0) v = ldexp((double)m, -24);
    else if (e == 31) v = m ? NAN : INFINITY;
    else v = ldexp(1024.0 + m, e - 25);
    return s ? -v : v;
}

uint16_t orc_f32_to_bf16(float x) {
    uint32_t bits;
    memcpy(&bits, &x, 4);
    uint16_t sign = (uint16_t)((bits >> 16) & 0x8000u);
    if (isnan(x)) return (uint16_t)(sign | 0x7fc0u);
    double ax = fabs((double)x);
    double v = round_to_format(ax, 7, -126);
    if (isinf(x) || v >= ldexp(1.0, 128)) return (uint16_t)(sign | 0x7f80u);
    if (v == 0.0) return sign;
    if (v < ldexp(1.0, -126)) return (uint16_t)(sign | (uint16_t)(v / ldexp(1.0, -133)));
    int e;
    frexp(v, &e);
    e -= 1;
    uint16_t m = (uint16_t)(v / ldexp(1.0, e - 7) - 128.0);
    return (uint16_t)(sign | (uint16_t)((e + 127) << 7) | m);
}

double orc_bf16_to_f64(uint16_t h) {
    uint32_t bits = (uint32_t)h << 16;
    float f;
    memcpy(&f, &bits, 4);
    return (double)f;
}

/* saturating: magnitudes that round above 448 become 448 */
uint8_t orc_f32_to_e4m3(float x) {
    uint32_t bits;
    memcpy(&bits, &x, 4);
    uint8_t sign = (uint8_t)((bits >> 24) & 0x80u);
    if (isnan(x)) return (uint8_t)(sign | 0x7fu);
    double ax = fabs((double)x);
    double v = round_to_format(ax, 3, -6);
    if (v > 448.0) v = 448.0;
    if (v == 0.0) return sign;
    if (v < ldexp(1.0, -6)) return (uint8_t)(sign | (uint8_t)(v / ldexp(1.0, -9)));
    int e;
    frexp(v, &e);
    e -= 1;
    uint8_t m = (uint8_t)(v / ldexp(1.0, e - 3) - 8.0);
    return (uint8_t)(sign | (uint8_t)((e + 7) << 3) | m);
}

double orc_e4m3_to_f64(uint8_t b) {
    int s = (b >> 7) & 1, e = (b >> 3) & 15, m = b & 7;
    double v;
    if (e == 15 && m == 7) v = NAN;
    else if (e == 0) v = ldexp((double)m, -9);
    else v = ldexp(8.0 + m, e - 10);
    return s ? -v : v;
}

/* Per-channel power-of-two scale exponent for FP8 storage: the smallest e
 * with amax <= 448 * 2^e (e = 0 for an all-zero channel). */
int32_t orc_e4m3_scale_exp(float amax) {
    if (!(amax > 0.0f)) return 0;
    int e;
    frexp((double)amax, &e);
    e -= 10;                        /* 448 * 2^(e) is below amax here */
    while ((double)amax > ldexp(448.0, e)) e++;
    while (e > -200 && (double)amax <= ldexp(448.0, e - 1)) e--;
    return e;
}

/* dtype: 0 fp32, 1 fp16, 2 bf16, 3 fp8-e4m3.  x holds n values; inv_scale[c]
 * (power of two) multiplies channel c = index % 8 before rounding; out_bits
 * receives the encoded values (4, 2, 2 or 1 bytes each) and out_deq the
 * decoded value times the channel scale (as float; exact for all formats). */
void orc_quantize(const float *x, int64_t n, int32_t dtype, const int32_t *scale_exp,
                  void *out_bits, float *out_deq) {
#pragma omp parallel for schedule(static)
    for (int64_t i = 0; i < n; i++) {
        int c = (int)(i % NCH);
        int se = scale_exp ? scale_exp[c] : 0;
        float xs = (float)ldexp((double)x[i], -se);
        double v;
        switch (dtype) {
        case 1: {
            uint16_t h = orc_f32_to_f16(xs);
            if (out_bits) ((uint16_t *)out_bits)[i] = h;
            v = orc_f16_to_f64(h);
            break;
        }
        case 2: {
            uint16_t h = orc_f32_to_bf16(xs);
            if (out_bits) ((uint16_t *)out_bits)[i] = h;
            v = orc_bf16_to_f64(h);
            break;
        }
        case 3: {
            uint8_t h = orc_f32_to_e4m3(xs);
            if (out_bits) ((uint8_t *)out_bits)[i] = h;
            v = orc_e4m3_to_f64(h);
            break;
        }
        default:
            if (out_bits) ((float *)out_bits)[i] = xs;
            v = (double)xs;
        }
        if (out_deq) out_deq[i] = (float)ldexp(v, se);
    }
}

/* ------------------------------------------------------------------------- */
/* FP32 decision sequence.  Every line is one IEEE-754 binary32 operation with
 * round-to-nearest-even; the file is compiled without contraction. */

static double focal_length(int32_t H, double fov_y_deg) {
    return (0.5 * (double)H) / tan(0.5 * fov_y_deg * M_PI / 180.0);
}

/* Pinhole ray through the centre of pixel (px, py): o = camera centre,
 * d = normalize(R * ((x+1/2-W/2)/f, -(y+1/2-H/2)/f, -1)). */
void orc_pixel_ray(const orc_camera *cam, int32_t px, int32_t py, float o[3], float d[3]) {
    const float f = (float)focal_length(cam->height, cam->fov_y_deg);
    const float bx = ((float)px + 0.5f) - 0.5f * (float)cam->width;
    const float by = ((float)py + 0.5f) - 0.5f * (float)cam->height;
    const float xc = bx / f;
    const float yc = -(by / f);
    float dw[3];
    for (int r = 0; r < 3; r++) {
        const float r0 = (float)cam->c2w[4 * r + 0];
        const float r1 = (float)cam->c2w[4 * r + 1];
        const float r2 = (float)cam->c2w[4 * r + 2];
        const float a = r0 * xc;
        const float b = r1 * yc;
        const float s = a + b;
        dw[r] = s - r2; /* times z_cam = -1 */
        o[r] = (float)cam->c2w[4 * r + 3];
    }
    const float n2 = (dw[0] * dw[0] + dw[1] * dw[1]) + dw[2] * dw[2];
    const float n = sqrtf(n2);
    for (int r = 0; r < 3; r++) d[r] = dw[r] / n;
}

/* Sample spacing of a block: the x side over the plane resolution. */
static float block_delta(const orc_block *b) {
    return (float)(((double)b->hi[0] - (double)b->lo[0]) / (double)b->P);
}

/* Lattice point i of a ray: t_i = (i + 1/2) delta, p = o + t_i d. */
static void lattice_point(const float o[3], const float d[3], float delta, int64_t i, float p[3]) {
    const float t = ((float)i + 0.5f) * delta;
    for (int a = 0; a < 3; a++) {
        const float td = t * d[a];
        p[a] = o[a] + td;
    }
}

/* Eq. 4 with half-open xy extents: a point belongs to the block whose
 * [lo, hi) x [lo, hi) footprint contains it; z is the closed [lo, hi]. */
static int inside_block(const orc_block *b, const float p[3]) {
    return p[0] >= b->lo[0] && p[0] < b->hi[0] && p[1] >= b->lo[1] && p[1] < b->hi[1] &&
           p[2] >= b->lo[2] && p[2] <= b->hi[2];
}

int32_t orc_occ_cells(int32_t R, int32_t C) { return (R - 1 + C - 1) / C; }

/* Threads of the oracle's parallel loops (for timing it on one core);
 * returns the new maximum. */
int32_t orc_set_threads(int32_t n) {
    if (n > 0) omp_set_num_threads(n);
    return omp_get_max_threads();
}

/* Occupancy cell of a point inside block b: the voxel v = floor(g) of the
 * continuous grid coordinate g = (p - lo) * ((R-1)/(hi-lo)), clamped to
 * [0, R-2], divided by the cell edge C. */
static int64_t occ_cell_index(const orc_block *b, const float p[3]) {
    const int Nc = orc_occ_cells(b->R, b->occ_cell);
    int cell[3];
    for (int a = 0; a < 3; a++) {
        const float k = (float)((double)(b->R - 1) / ((double)b->hi[a] - (double)b->lo[a]));
        const float rel = p[a] - b->lo[a];
        const float g = rel * k;
        int v = (int)floorf(g);
        if (v < 0) v = 0;
        if (v > b->R - 2) v = b->R - 2;
        cell[a] = v / b->occ_cell;
    }
    return ((int64_t)cell[2] * Nc + cell[1]) * Nc + cell[0];
}

static int occupied(const orc_block *b, const float p[3]) {
    if (!b->occ) return 1;
    int64_t c = occ_cell_index(b, p);
    return (int)((b->occ[c >> 5] >> (c & 31)) & 1u);
}

/* Occupancy grid: the bit of cell (cx, cy, cz) is set when any grid vertex
 * in [C*c, C*c + C] (clamped to R-1) along every axis has density
 * exp(ch0) > thresh, i.e. ch0 > ln(thresh) decided in double. */
void orc_occupancy(const float *grid, int32_t R, int32_t C, float thresh, uint32_t *bits) {
    const int Nc = orc_occ_cells(R, C);
    const int64_t ncell = (int64_t)Nc * Nc * Nc;
    memset(bits, 0, (size_t)((ncell + 31) / 32) * 4);
    const double lt = log((double)thresh);
#pragma omp parallel for schedule(dynamic, 1)
    for (int cz = 0; cz < Nc; cz++)
        for (int cy = 0; cy < Nc; cy++)
            for (int cx = 0; cx < Nc; cx++) {
                int on = 0;
                for (int z = cz * C; z <= cz * C + C && z < R && !on; z++)
                    for (int y = cy * C; y <= cy * C + C && y < R && !on; y++)
                        for (int x = cx * C; x <= cx * C + C && x < R && !on; x++)
                            if ((double)grid[(((int64_t)z * R + y) * R + x) * NCH] > lt) on = 1;
                if (on) {
                    int64_t c = ((int64_t)cz * Nc + cy) * Nc + cx;
#pragma omp atomic
                    bits[c >> 5] |= 1u << (c & 31);
                }
            }
}

/* ------------------------------------------------------------------------- */
/* Feature lookup f^{k,l}(p): trilinear grid + bilinear xy, xz, yz planes.   */

typedef struct taps {
    int64_t gidx[8];   /* element offsets of the 8 grid vertices (channel 0) */
    double gw[8];
    int64_t pidx[3][4];
    double pw[3][4];
} taps;

static double load_el(const void *base, int is_f64, int64_t idx) {
    return is_f64 ? ((const double *)base)[idx] : (double)((const float *)base)[idx];
}

/* vertex-aligned coordinate: vertex 0 at lo, vertex n-1 at hi */
static void axis_coord(double p, double lo, double hi, int n, int *c0, double *fr) {
    double g = (p - lo) * (double)(n - 1) / (hi - lo);
    if (g < 0.0) g = 0.0;
    if (g > (double)(n - 1)) g = (double)(n - 1);
    int c = (int)floor(g);
    if (c > n - 2) c = n - 2;
    *c0 = c;
    *fr = g - (double)c;
}

static void make_taps(const orc_block *b, const double p[3], taps *tp) {
    int c[3];
    double fr[3];
    for (int a = 0; a < 3; a++) axis_coord(p[a], b->lo[a], b->hi[a], b->R, &c[a], &fr[a]);
    const int64_t R = b->R;
    int k = 0;
    for (int dz = 0; dz < 2; dz++)
        for (int dy = 0; dy < 2; dy++)
            for (int dx = 0; dx < 2; dx++, k++) {
                tp->gidx[k] = (((c[2] + dz) * R + (c[1] + dy)) * R + (c[0] + dx)) * NCH;
                tp->gw[k] = (dx ? fr[0] : 1.0 - fr[0]) * (dy ? fr[1] : 1.0 - fr[1]) *
                            (dz ? fr[2] : 1.0 - fr[2]);
            }
    int h[3];
    double hf[3];
    for (int a = 0; a < 3; a++) axis_coord(p[a], b->lo[a], b->hi[a], b->P, &h[a], &hf[a]);
    static const int pu[3] = {0, 0, 1}, pv[3] = {1, 2, 2}; /* xy, xz, yz */
    const int64_t P = b->P;
    for (int pl = 0; pl < 3; pl++) {
        int u = h[pu[pl]], v = h[pv[pl]];
        double fu = hf[pu[pl]], fv = hf[pv[pl]];
        int q = 0;
        for (int dv = 0; dv < 2; dv++)
            for (int du = 0; du < 2; du++, q++) {
                tp->pidx[pl][q] = ((v + dv) * P + (u + du)) * NCH;
                tp->pw[pl][q] = (du ? fu : 1.0 - fu) * (dv ? fv : 1.0 - fv);
            }
    }
}

/* Taps of a contracted block at contracted coordinates u in [-2, 2]^3. */
static void make_taps_u(const orc_block *b, const double u[3], taps *tp) {
    orc_block v = *b;
    for (int a = 0; a < 3; a++) {
        v.lo[a] = -2.0f;
        v.hi[a] = 2.0f;
    }
    make_taps(&v, u, tp);
}

static void eval_feature(const orc_block *b, const taps *tp, double f[NCH]) {
    for (int c = 0; c < NCH; c++) f[c] = 0.0;
    for (int k = 0; k < 8; k++)
        for (int c = 0; c < NCH; c++) f[c] += tp->gw[k] * load_el(b->grid, b->is_f64, tp->gidx[k] + c);
    for (int pl = 0; pl < 3; pl++)
        for (int q = 0; q < 4; q++)
            for (int c = 0; c < NCH; c++)
                f[c] += tp->pw[pl][q] * load_el(b->planes[pl], b->is_f64, tp->pidx[pl][q] + c);
}

double orc_feature_at(const orc_block *b, const double p[3], double *f) {
    taps tp;
    make_taps(b, p, &tp);
    eval_feature(b, &tp, f);
    return f[0];
}

static double sigmoid(double x) { return 1.0 / (1.0 + exp(-x)); }

/* ------------------------------------------------------------------------- */
/* Samples of one ray inside one block.                                      */

typedef struct sample {
    double t;          /* FP32 lattice t, as double */
    double alpha;      /* 1 - exp(-sigma delta) */
    double sigma;
    double delta;
    double c[3];       /* sigmoid(f1..3) */
    double s[4];       /* sigmoid(f4..7) */
    int32_t block;     /* index into the block array */
    taps tp;
} sample;

typedef struct sample_vec {
    sample *v;
    int64_t n, cap;
} sample_vec;

static void push_sample(sample_vec *sv, const sample *s) {
    if (sv->n == sv->cap) {
        sv->cap = sv->cap ? 2 * sv->cap : 256;
        sv->v = (sample *)realloc(sv->v, (size_t)sv->cap * sizeof(sample));
    }
    sv->v[sv->n++] = *s;
}

/* Candidate lattice indices of block b: the FP64 slab interval of the box
 * grown by a margin far above FP32 position error (1e-3 of the block
 * extent), widened by one index at each end.  Any lattice point whose FP32
 * position lies in the box lies in this range; membership itself is decided
 * by inside_block on the FP32 point. */
static int candidate_range(const orc_block *b, const float of[3], const float df[3], float delta,
                           int64_t *i0, int64_t *i1) {
    double tn = 0.0, tf = INFINITY;
    for (int a = 0; a < 3; a++) {
        const double ext = (double)b->hi[a] - (double)b->lo[a];
        const double m = 1e-3 * (ext > 1.0 ? ext : 1.0);
        const double lo = (double)b->lo[a] - m, hi = (double)b->hi[a] + m;
        const double o = of[a], d = df[a];
        if (d == 0.0) {
            if (o < lo || o > hi) return 0;
            continue;
        }
        double t0 = (lo - o) / d, t1 = (hi - o) / d;
        if (t0 > t1) {
            double tmp = t0;
            t0 = t1;
            t1 = tmp;
        }
        if (t0 > tn) tn = t0;
        if (t1 < tf) tf = t1;
    }
    if (!(tn <= tf)) return 0;
    const double dl = (double)delta;
    int64_t a0 = (int64_t)floor(tn / dl - 0.5) - 1;
    int64_t a1 = (int64_t)ceil(tf / dl - 0.5) + 1;
    if (a0 < 0) a0 = 0;
    if (a1 < a0) return 0;
    *i0 = a0;
    *i1 = a1;
    return 1;
}

/* ------------------------------------------------------------------------- */
/* Unbounded (contracted) boundary blocks.  Implementation details of the
 * paper: blocks on the scene's boundary hold an unbounded representation
 * with MERF's contraction (Eq. 16), which maps the space outside the unit
 * cube of the block's normalised coordinates x = (p - c) / h (c the centre
 * and h the half extents of its box) into the shell 1 < ||u||_inf < 2.  The
 * grid and planes of such a block span u in [-2, 2]^3.
 *
 * The block owns its xy footprint extended to infinity across the sides
 * flagged in `unbounded` (the sides on the scene's boundary), half-open as
 * in Eq. 4, and every z.  A ray is marched through it from its first
 * standard lattice point inside that region with the FP32 recurrence
 * t_{k+1} = t_k + s_k, s_k = (delta m) m, m = max(1, ||x(t_k)||_inf): one
 * lattice step inside the box and, outside, one lattice step of the
 * dominant contracted coordinate (d/dm (2 - 1/m) = 1/m^2).  Sample k's
 * opacity is 1 - exp(-sigma s_k).  The march stops when the point leaves
 * the region, when ||x||_inf > 1e4, or after 65536 steps.  Decisions use the
 * FP32 sequence below; interpolation is FP64 at the FP32 sample point. */

static int owned_unbounded(const orc_block *b, const float p[3]) {
    const int e = b->unbounded;
    return ((e & ORC_EXT_XLO) || p[0] >= b->lo[0]) && ((e & ORC_EXT_XHI) || p[0] < b->hi[0]) &&
           ((e & ORC_EXT_YLO) || p[1] >= b->lo[1]) && ((e & ORC_EXT_YHI) || p[1] < b->hi[1]);
}

/* FP32 normalised coordinates and their infinity norm. */
static float contract_x32(const orc_block *b, const float p[3], float x[3]) {
    float m = 0.0f;
    for (int a = 0; a < 3; a++) {
        const float c = (float)(0.5 * ((double)b->lo[a] + (double)b->hi[a]));
        const float ih = (float)(2.0 / ((double)b->hi[a] - (double)b->lo[a]));
        const float rel = p[a] - c;
        x[a] = rel * ih;
        const float ax = fabsf(x[a]);
        if (ax > m) m = ax;
    }
    return m;
}

/* Eq. 16 in FP32: u_j = x_j inside the unit cube; outside, 2 - 1/|x_j| (with
 * x_j's sign) on the coordinates that reach the norm, x_j / m on the rest. */
static void contract_u32(const float x[3], float m, float u[3]) {
    for (int a = 0; a < 3; a++) {
        if (m <= 1.0f) {
            u[a] = x[a];
        } else if (fabsf(x[a]) == m) {
            const float q = 1.0f / fabsf(x[a]);
            const float v = 2.0f - q;
            u[a] = x[a] < 0.0f ? -v : v;
        } else {
            u[a] = x[a] / m;
        }
    }
}

/* Eq. 16 in FP64 (interpolation). */
void orc_contract(const double x[3], double u[3]) {
    double m = 0.0;
    for (int a = 0; a < 3; a++)
        if (fabs(x[a]) > m) m = fabs(x[a]);
    for (int a = 0; a < 3; a++) {
        if (m <= 1.0) u[a] = x[a];
        else if (fabs(x[a]) == m) u[a] = (2.0 - 1.0 / fabs(x[a])) * (x[a] < 0.0 ? -1.0 : 1.0);
        else u[a] = x[a] / m;
    }
}

static int occupied_unbounded(const orc_block *b, const float u[3]) {
    if (!b->occ) return 1;
    const int Nc = orc_occ_cells(b->R, b->occ_cell);
    const float k = (float)((double)(b->R - 1) / 4.0);
    int cell[3];
    for (int a = 0; a < 3; a++) {
        const float s = u[a] + 2.0f;
        const float g = s * k;
        int v = (int)floorf(g);
        if (v < 0) v = 0;
        if (v > b->R - 2) v = b->R - 2;
        cell[a] = v / b->occ_cell;
    }
    const int64_t c = ((int64_t)cell[2] * Nc + cell[1]) * Nc + cell[0];
    return (int)((b->occ[c >> 5] >> (c & 31)) & 1u);
}

static void make_taps(const orc_block *b, const double p[3], taps *tp);
static void make_taps_u(const orc_block *b, const double u[3], taps *tp);

/* First lattice index of the ray inside the block's region, or -1.  The
 * region is convex and each FP32 lattice coordinate is monotone in the
 * index, so the owned indices form one interval; its start is found from the
 * FP32 entry estimate j = floor(t_in / delta - 1/2) of the bounded xy sides
 * by stepping back while the previous point is owned, or forward (at most
 * 64 points) until one is.  Every operation is FP32 round-to-nearest. */
static int64_t first_owned_index(const orc_block *b, const float of[3], const float df[3], float delta) {
    float tn = 0.0f;
    for (int a = 0; a < 2; a++) {
        const int elo = b->unbounded & (a == 0 ? ORC_EXT_XLO : ORC_EXT_YLO);
        const int ehi = b->unbounded & (a == 0 ? ORC_EXT_XHI : ORC_EXT_YHI);
        if (df[a] == 0.0f) {
            if ((!elo && of[a] < b->lo[a]) || (!ehi && of[a] >= b->hi[a])) return -1;
            continue;
        }
        const float inv = 1.0f / df[a];
        const float bound = df[a] > 0.0f ? b->lo[a] : b->hi[a];
        if (df[a] > 0.0f ? elo : ehi) continue;
        const float rel = bound - of[a];
        const float te = rel * inv;
        if (te > tn) tn = te;
    }
    const float inv_delta = 1.0f / delta;
    const float xq = tn * inv_delta;
    const float xs = xq - 0.5f;
    if (!(xs < 16777216.0f)) return -1;
    int64_t j = (int64_t)floorf(xs);
    if (j < 0) j = 0;
    float p[3];
    lattice_point(of, df, delta, j, p);
    if (owned_unbounded(b, p)) {
        for (int k = 0; k < 64 && j > 0; k++) {
            lattice_point(of, df, delta, j - 1, p);
            if (!owned_unbounded(b, p)) break;
            j--;
        }
        return j;
    }
    for (int k = 1; k <= 64; k++) {
        lattice_point(of, df, delta, j + k, p);
        if (owned_unbounded(b, p)) return j + k;
    }
    return -1;
}

static int64_t unbounded_samples(const orc_block *blocks, int32_t bi, const float of[3], const float df[3],
                                 sample_vec *out) {
    const orc_block *b = &blocks[bi];
    const float delta = block_delta(b);
    const int64_t i0 = first_owned_index(b, of, df, delta);
    if (i0 < 0) return 0;
    float t = ((float)i0 + 0.5f) * delta;
    int64_t n = 0;
    for (int k = 0; k < ORC_CONTRACT_STEPS; k++) {
        float pf[3];
        for (int a = 0; a < 3; a++) {
            const float td = t * df[a];
            pf[a] = of[a] + td;
        }
        if (!owned_unbounded(b, pf)) break;
        float x[3];
        const float m = contract_x32(b, pf, x);
        if (m > ORC_CONTRACT_MAX) break;
        const float m1 = m > 1.0f ? m : 1.0f;
        const float dm = delta * m1;
        const float step = dm * m1;
        float u[3];
        contract_u32(x, m, u);
        if (occupied_unbounded(b, u)) {
            sample s;
            double x64[3], u64[3];
            for (int a = 0; a < 3; a++) {
                const double c = 0.5 * ((double)b->lo[a] + (double)b->hi[a]);
                const double h = 0.5 * ((double)b->hi[a] - (double)b->lo[a]);
                x64[a] = ((double)pf[a] - c) / h;
            }
            orc_contract(x64, u64);
            make_taps_u(b, u64, &s.tp);
            double f[NCH];
            eval_feature(b, &s.tp, f);
            s.t = (double)t;
            s.delta = (double)step;
            s.sigma = exp(f[0]);
            s.alpha = -expm1(-s.sigma * s.delta);
            for (int c = 0; c < 3; c++) s.c[c] = sigmoid(f[1 + c]);
            for (int c = 0; c < 4; c++) s.s[c] = sigmoid(f[4 + c]);
            s.block = bi;
            push_sample(out, &s);
            n++;
        }
        t = t + step;
    }
    return n;
}

/* Append the occupied samples of block bi along the ray, in lattice order;
 * returns the number appended. */
static int64_t block_samples(const orc_block *blocks, int32_t bi, const float of[3], const float df[3],
                             sample_vec *out) {
    const orc_block *b = &blocks[bi];
    if (b->unbounded & ORC_CONTRACTED) return unbounded_samples(blocks, bi, of, df, out);
    const float delta = block_delta(b);
    int64_t i0, i1, n = 0;
    if (!candidate_range(b, of, df, delta, &i0, &i1)) return 0;
    for (int64_t i = i0; i <= i1; i++) {
        float pf[3];
        lattice_point(of, df, delta, i, pf);
        if (!inside_block(b, pf)) continue;
        if (!occupied(b, pf)) continue; /* empty cells are skipped (Sec. 4.5) */
        sample s;
        const double p[3] = {pf[0], pf[1], pf[2]};
        make_taps(b, p, &s.tp);
        double f[NCH];
        eval_feature(b, &s.tp, f);
        s.t = (double)(((float)i + 0.5f) * delta);
        s.delta = (double)delta;
        s.sigma = exp(f[0]);
        s.alpha = -expm1(-s.sigma * s.delta); /* Eq. 1 */
        for (int c = 0; c < 3; c++) s.c[c] = sigmoid(f[1 + c]);
        for (int c = 0; c < 4; c++) s.s[c] = sigmoid(f[4 + c]);
        s.block = bi;
        push_sample(out, &s);
        n++;
    }
    return n;
}

/* ------------------------------------------------------------------------- */
/* Deferred MLP (Eq. 3): x = [C_d, F, d] -> 16 ReLU -> 16 ReLU -> 3 sigmoid,
 * C = C_d + Phi(x).  Weights are input-major: W1[i][j] at OFF_W1 + i*16 + j. */

typedef struct mlp_trace {
    double x[MLP_IN], z1[MLP_HID], h1[MLP_HID], z2[MLP_HID], h2[MLP_HID], z3[MLP_OUT], o[MLP_OUT];
} mlp_trace;

static void mlp_forward(const double *w, const double x[MLP_IN], mlp_trace *tr) {
    memcpy(tr->x, x, sizeof(tr->x));
    for (int j = 0; j < MLP_HID; j++) {
        double a = w[OFF_B1 + j];
        for (int i = 0; i < MLP_IN; i++) a += x[i] * w[OFF_W1 + i * MLP_HID + j];
        tr->z1[j] = a;
        tr->h1[j] = a > 0.0 ? a : 0.0;
    }
    for (int j = 0; j < MLP_HID; j++) {
        double a = w[OFF_B2 + j];
        for (int i = 0; i < MLP_HID; i++) a += tr->h1[i] * w[OFF_W2 + i * MLP_HID + j];
        tr->z2[j] = a;
        tr->h2[j] = a > 0.0 ? a : 0.0;
    }
    for (int j = 0; j < MLP_OUT; j++) {
        double a = w[OFF_B3 + j];
        for (int i = 0; i < MLP_HID; i++) a += tr->h2[i] * w[OFF_W3 + i * MLP_OUT + j];
        tr->z3[j] = a;
        tr->o[j] = sigmoid(a);
    }
}

void orc_mlp(const double *w, const double *x, int64_t n, double *out) {
    for (int64_t r = 0; r < n; r++) {
        mlp_trace tr;
        mlp_forward(w, x + r * MLP_IN, &tr);
        for (int j = 0; j < MLP_OUT; j++) out[r * MLP_OUT + j] = tr.o[j];
    }
}

/* ------------------------------------------------------------------------- */
/* One ray.                                                                  */

enum { MODE_BLOCKWISE = 0, MODE_SINGLE_PASS = 1, MODE_ALPHA_NORM = 2 };

typedef struct ray_result {
    double rgb[3];
    double aux[8]; /* C_d (3), F (4), transmittance left after the last block */
    int32_t nsamp;
} ray_result;

static int cmp_sample_t(const void *a, const void *b) {
    const sample *x = (const sample *)a, *y = (const sample *)b;
    if (x->t < y->t) return -1;
    if (x->t > y->t) return 1;
    return 0;
}

/* Composite the samples (already grouped per block in `order`) by `mode`;
 * seg[k]..seg[k+1] delimits the samples of the k-th block in order. */
static void composite(const sample_vec *sv, const int64_t *seg, int32_t nseg, int32_t mode,
                      double Cd[3], double F[4], double *Tout) {
    for (int c = 0; c < 3; c++) Cd[c] = 0.0;
    for (int c = 0; c < 4; c++) F[c] = 0.0;
    if (mode == MODE_SINGLE_PASS) {
        /* Eq. 1-2 (= Eq. 14 of Appendix A) over the merged samples in depth order */
        sample *tmp = (sample *)malloc((size_t)(sv->n ? sv->n : 1) * sizeof(sample));
        memcpy(tmp, sv->v, (size_t)sv->n * sizeof(sample));
        qsort(tmp, (size_t)sv->n, sizeof(sample), cmp_sample_t);
        double T = 1.0;
        for (int64_t i = 0; i < sv->n; i++) {
            const double w = T * tmp[i].alpha;
            for (int c = 0; c < 3; c++) Cd[c] += w * tmp[i].c[c];
            for (int c = 0; c < 4; c++) F[c] += w * tmp[i].s[c];
            T *= 1.0 - tmp[i].alpha;
        }
        *Tout = T;
        free(tmp);
        return;
    }
    /* Eq. 11: per block colour C_d^k, feature F^k and opacity alpha^k */
    double Ck[64][3], Fk[64][4], Ak[64];
    double(*pCk)[3] = Ck;
    double(*pFk)[4] = Fk;
    double *pAk = Ak;
    if (nseg > 64) {
        pCk = (double(*)[3])malloc((size_t)nseg * sizeof(*pCk));
        pFk = (double(*)[4])malloc((size_t)nseg * sizeof(*pFk));
        pAk = (double *)malloc((size_t)nseg * sizeof(double));
    }
    for (int k = 0; k < nseg; k++) {
        double c3[3] = {0, 0, 0}, f4[4] = {0, 0, 0, 0}, a = 0.0;
        double T = 1.0; /* prod_{j<i} (1 - alpha_j) within the block */
        for (int64_t i = seg[k]; i < seg[k + 1]; i++) {
            const double w = T * sv->v[i].alpha; /* w_i of Eq. 11 */
            for (int c = 0; c < 3; c++) c3[c] += w * sv->v[i].c[c];
            for (int c = 0; c < 4; c++) f4[c] += w * sv->v[i].s[c];
            a += w;
            T *= 1.0 - sv->v[i].alpha;
        }
        memcpy(pCk[k], c3, sizeof(c3));
        memcpy(pFk[k], f4, sizeof(f4));
        pAk[k] = a;
    }
    if (mode == MODE_ALPHA_NORM) {
        /* ablation "no alpha blending": blocks weighted by alpha^k / sum_j alpha^j */
        double sa = 0.0, T = 1.0;
        for (int k = 0; k < nseg; k++) sa += pAk[k];
        for (int k = 0; k < nseg; k++) {
            const double wk = sa > 0.0 ? pAk[k] / sa : 0.0;
            for (int c = 0; c < 3; c++) Cd[c] += wk * pCk[k][c];
            for (int c = 0; c < 4; c++) F[c] += wk * pFk[k][c];
            T *= 1.0 - pAk[k];
        }
        *Tout = T;
    } else {
        /* Eq. 5 / Eq. 12: C = sum_k prod_{j<k} (1 - alpha^j) C^k */
        for (int k = 0; k < nseg; k++) {
            double Tk = 1.0;
            for (int j = 0; j < k; j++) Tk *= 1.0 - pAk[j];
            for (int c = 0; c < 3; c++) Cd[c] += Tk * pCk[k][c];
            for (int c = 0; c < 4; c++) F[c] += Tk * pFk[k][c];
        }
        double T = 1.0;
        for (int k = 0; k < nseg; k++) T *= 1.0 - pAk[k];
        *Tout = T;
    }
    if (nseg > 64) {
        free(pCk);
        free(pFk);
        free(pAk);
    }
}

static void render_one_ray(const orc_block *blocks, const int32_t *order, int32_t n_order,
                           const float of[3], const float df[3], const double *mlp, int32_t mode,
                           ray_result *res, sample_vec *sv, int64_t **segbuf, int32_t *segcap) {
    sv->n = 0;
    if (*segcap < n_order + 1) {
        *segcap = n_order + 1;
        *segbuf = (int64_t *)realloc(*segbuf, (size_t)(*segcap) * sizeof(int64_t));
    }
    int64_t *seg = *segbuf;
    seg[0] = 0;
    for (int k = 0; k < n_order; k++) {
        block_samples(blocks, order[k], of, df, sv);
        seg[k + 1] = sv->n;
    }
    double Cd[3], F[4], T;
    composite(sv, seg, n_order, mode, Cd, F, &T);
    for (int c = 0; c < 3; c++) res->aux[c] = Cd[c];
    for (int c = 0; c < 4; c++) res->aux[3 + c] = F[c];
    res->aux[7] = T;
    res->nsamp = (int32_t)sv->n;
    if (mlp) {
        double x[MLP_IN] = {Cd[0], Cd[1], Cd[2], F[0], F[1], F[2], F[3], df[0], df[1], df[2]};
        mlp_trace tr;
        mlp_forward(mlp, x, &tr);
        for (int c = 0; c < 3; c++) res->rgb[c] = Cd[c] + tr.o[c];
    } else {
        for (int c = 0; c < 3; c++) res->rgb[c] = Cd[c];
    }
}

/* Render pixels of one view.  order: block indices sorted near to far (from
 * orc_select_lod or the caller).  pix: linear pixel indices y*W + x (NULL =
 * every pixel, row-major).  mlp: 499 weights or NULL (output C_d). */
void orc_render_view(const orc_block *blocks, int32_t nb, const int32_t *order, int32_t n_order,
                     const orc_camera *cam, const double *mlp, int32_t mode, const int64_t *pix,
                     int64_t n_pix, double *out_rgb, double *out_aux, int32_t *out_nsamp) {
    (void)nb;
    const int64_t W = cam->width;
    const int64_t npx = pix ? n_pix : W * (int64_t)cam->height;
#pragma omp parallel
    {
        sample_vec sv = {0, 0, 0};
        int64_t *seg = NULL;
        int32_t segcap = 0;
#pragma omp for schedule(dynamic, 16)
        for (int64_t r = 0; r < npx; r++) {
            const int64_t lin = pix ? pix[r] : r;
            float of[3], df[3];
            orc_pixel_ray(cam, (int32_t)(lin % W), (int32_t)(lin / W), of, df);
            ray_result res;
            render_one_ray(blocks, order, n_order, of, df, mlp, mode, &res, &sv, &seg, &segcap);
            if (out_rgb)
                for (int c = 0; c < 3; c++) out_rgb[r * 3 + c] = res.rgb[c];
            if (out_aux)
                for (int c = 0; c < 8; c++) out_aux[r * 8 + c] = res.aux[c];
            if (out_nsamp) out_nsamp[r] = res.nsamp;
        }
        free(sv.v);
        free(seg);
    }
}

/* ------------------------------------------------------------------------- */
/* Per-block deferred MLPs (Sec. 4.1 rendering stage: every block k of LOD l
 * carries its own tiny MLP Phi^{k,l}; Sec. 4.2: each block's colour C^k is
 * Eq. 3 applied to that block's own C_d^k and F^k, and the block colours are
 * blended near to far by Eq. 5).  The MLP input is [C_d^k, F^k, PE(d)].
 *
 * PE(d) with L frequencies: d itself, then for l = 0 .. L-1 the three values
 * sin(2^l d) followed by the three values cos(2^l d) (component order x, y,
 * z); L = 0 gives the plain direction of the global form.  Weights of a
 * block MLP are input-major like the global one: W1[n_in][16], b1[16],
 * W2[16][16], b2[16], W3[16][3], b3[3], n_in = 7 + 3 + 6 L.
 *
 * A block takes part in Eq. 5 when the ray has at least one occupied sample
 * in it; a block the ray crosses only through empty cells adds nothing (its
 * C_d^k, F^k and alpha^k are zero, and Phi^k of empty features is not a
 * colour of that block). */

int32_t orc_pe_dim(int32_t L) { return 3 + 6 * L; }

int32_t orc_block_mlp_nparam(int32_t L) {
    const int32_t n_in = 7 + orc_pe_dim(L);
    return n_in * MLP_HID + MLP_HID + MLP_HID * MLP_HID + MLP_HID + MLP_HID * MLP_OUT + MLP_OUT;
}

void orc_pe(const double d[3], int32_t L, double *out) {
    for (int a = 0; a < 3; a++) out[a] = d[a];
    double f = 1.0; /* 2^l */
    for (int32_t l = 0; l < L; l++) {
        for (int a = 0; a < 3; a++) out[3 + 6 * l + a] = sin(f * d[a]);
        for (int a = 0; a < 3; a++) out[3 + 6 * l + 3 + a] = cos(f * d[a]);
        f *= 2.0;
    }
}

/* Phi of Eq. 3 for an n_in-input MLP: ReLU, ReLU, sigmoid. */
static void mlp_n(const double *w, int32_t n_in, const double *x, double out[MLP_OUT]) {
    const double *W1 = w, *b1 = W1 + n_in * MLP_HID, *W2 = b1 + MLP_HID, *b2 = W2 + MLP_HID * MLP_HID;
    const double *W3 = b2 + MLP_HID, *b3 = W3 + MLP_HID * MLP_OUT;
    double h1[MLP_HID], h2[MLP_HID];
    for (int j = 0; j < MLP_HID; j++) {
        double a = b1[j];
        for (int i = 0; i < n_in; i++) a += x[i] * W1[i * MLP_HID + j];
        h1[j] = a > 0.0 ? a : 0.0;
    }
    for (int j = 0; j < MLP_HID; j++) {
        double a = b2[j];
        for (int i = 0; i < MLP_HID; i++) a += h1[i] * W2[i * MLP_HID + j];
        h2[j] = a > 0.0 ? a : 0.0;
    }
    for (int j = 0; j < MLP_OUT; j++) {
        double a = b3[j];
        for (int i = 0; i < MLP_HID; i++) a += h2[i] * W3[i * MLP_OUT + j];
        out[j] = sigmoid(a);
    }
}

/* One ray with per-block MLPs (Sec. 4.1 Phi^{k,l}; Eq. 11 in-block weights,
 * Eq. 3 per block, Eq. 5 blend near to far over `order`).  x: scratch of
 * 7 + pe_dim(L) doubles.  Writes rgb (3), aux (C_d, F blended by Eq. 12 and
 * the transmittance after the last block) and the occupied-sample count. */
static void render_one_ray_block_mlp(const orc_block *blocks, const int32_t *order, int32_t n_order,
                                     const float of[3], const float df[3], const double *mlps, int32_t L,
                                     double *x, sample_vec *sv, double rgb[3], double aux[8], int32_t *nsamp) {
    const int32_t n_in = 7 + orc_pe_dim(L), np = orc_block_mlp_nparam(L);
    const double d[3] = {df[0], df[1], df[2]};
    double C[3] = {0, 0, 0}, Cd[3] = {0, 0, 0}, F[4] = {0, 0, 0, 0};
    double Tb = 1.0; /* prod_{j<k} (1 - alpha^j) */
    int32_t ns = 0;
    for (int k = 0; k < n_order; k++) {
        sv->n = 0;
        const int64_t nk = block_samples(blocks, order[k], of, df, sv);
        if (nk == 0) continue;
        /* Eq. 11: C_d^k, F^k, alpha^k with in-block weights */
        double ck[3] = {0, 0, 0}, fk[4] = {0, 0, 0, 0}, ak = 0.0, T = 1.0;
        for (int64_t i = 0; i < nk; i++) {
            const double w = T * sv->v[i].alpha;
            for (int c = 0; c < 3; c++) ck[c] += w * sv->v[i].c[c];
            for (int c = 0; c < 4; c++) fk[c] += w * sv->v[i].s[c];
            ak += w;
            T *= 1.0 - sv->v[i].alpha;
        }
        /* Eq. 3 with block k's MLP */
        for (int c = 0; c < 3; c++) x[c] = ck[c];
        for (int c = 0; c < 4; c++) x[3 + c] = fk[c];
        orc_pe(d, L, x + 7);
        double phi[MLP_OUT];
        mlp_n(mlps + (int64_t)order[k] * np, n_in, x, phi);
        /* Eq. 5 */
        for (int c = 0; c < 3; c++) C[c] += Tb * (ck[c] + phi[c]);
        for (int c = 0; c < 3; c++) Cd[c] += Tb * ck[c];
        for (int c = 0; c < 4; c++) F[c] += Tb * fk[c];
        Tb *= 1.0 - ak;
        ns += (int32_t)nk;
    }
    for (int c = 0; c < 3; c++) rgb[c] = C[c];
    for (int c = 0; c < 3; c++) aux[c] = Cd[c];
    for (int c = 0; c < 4; c++) aux[3 + c] = F[c];
    aux[7] = Tb;
    *nsamp = ns;
}

/* Render pixels of one view with per-block MLPs.  mlps: nb blocks' weights,
 * block i's at mlps + i * orc_block_mlp_nparam(L).  Outputs: rgb = Eq. 5;
 * aux = the blended C_d, F (Eq. 12) and the transmittance after the last
 * block; nsamp = occupied samples. */
void orc_render_view_block_mlp(const orc_block *blocks, int32_t nb, const int32_t *order, int32_t n_order,
                               const orc_camera *cam, const double *mlps, int32_t L, const int64_t *pix,
                               int64_t n_pix, double *out_rgb, double *out_aux, int32_t *out_nsamp) {
    (void)nb;
    const int64_t W = cam->width;
    const int64_t npx = pix ? n_pix : W * (int64_t)cam->height;
    const int32_t n_in = 7 + orc_pe_dim(L);
#pragma omp parallel
    {
        sample_vec sv = {0, 0, 0};
        double *x = (double *)malloc((size_t)n_in * sizeof(double));
#pragma omp for schedule(dynamic, 16)
        for (int64_t r = 0; r < npx; r++) {
            const int64_t lin = pix ? pix[r] : r;
            float of[3], df[3];
            orc_pixel_ray(cam, (int32_t)(lin % W), (int32_t)(lin / W), of, df);
            double rgb[3], aux[8];
            int32_t ns;
            render_one_ray_block_mlp(blocks, order, n_order, of, df, mlps, L, x, &sv, rgb, aux, &ns);
            if (out_rgb)
                for (int c = 0; c < 3; c++) out_rgb[r * 3 + c] = rgb[c];
            if (out_aux)
                for (int c = 0; c < 8; c++) out_aux[r * 8 + c] = aux[c];
            if (out_nsamp) out_nsamp[r] = ns;
        }
        free(sv.v);
        free(x);
    }
}

/* Block order for a ray with its own origin: Appendix D's xy distance from the
 * block centre to the origin, as the FP32 key (dx*dx + dy*dy) with
 * dx = cx - o_x, cx = (float)((lo_x + hi_x) / 2) in double; ties by index. */
static float ray_sort_key(const orc_block *b, const float o[3]) {
    const float cx = (float)(0.5 * ((double)b->lo[0] + (double)b->hi[0]));
    const float cy = (float)(0.5 * ((double)b->lo[1] + (double)b->hi[1]));
    const float dx = cx - o[0];
    const float dy = cy - o[1];
    return dx * dx + dy * dy;
}

static void sort_ids_for_ray(const orc_block *blocks, const int32_t *ids, int32_t n, const float o[3],
                             int32_t *out) {
    /* insertion sort on (key, id): plain and stable */
    float key[512];
    float *k = n <= 512 ? key : (float *)malloc((size_t)n * sizeof(float));
    for (int i = 0; i < n; i++) {
        int32_t id = ids[i];
        float kk = ray_sort_key(&blocks[id], o);
        int j = i - 1;
        while (j >= 0 && (k[j] > kk || (k[j] == kk && out[j] > id))) {
            k[j + 1] = k[j];
            out[j + 1] = out[j];
            j--;
        }
        k[j + 1] = kk;
        out[j + 1] = id;
    }
    if (k != key) free(k);
}

void orc_sort_ids_for_ray(const orc_block *blocks, const int32_t *ids, int32_t n, const float *o,
                          int32_t *out) {
    sort_ids_for_ray(blocks, ids, n, o, out);
}

/* Render independent rays (FP32 origins and unit directions, n x 3). */
void orc_render_rays(const orc_block *blocks, int32_t nb, const int32_t *ids, int32_t n_ids,
                     const float *o, const float *d, int64_t n_rays, const double *mlp, int32_t mode,
                     double *out_rgb, double *out_aux, int32_t *out_nsamp) {
    (void)nb;
#pragma omp parallel
    {
        sample_vec sv = {0, 0, 0};
        int64_t *seg = NULL;
        int32_t segcap = 0;
        int32_t *order = (int32_t *)malloc((size_t)(n_ids ? n_ids : 1) * sizeof(int32_t));
#pragma omp for schedule(dynamic, 16)
        for (int64_t r = 0; r < n_rays; r++) {
            sort_ids_for_ray(blocks, ids, n_ids, o + 3 * r, order);
            ray_result res;
            render_one_ray(blocks, order, n_ids, o + 3 * r, d + 3 * r, mlp, mode, &res, &sv, &seg, &segcap);
            if (out_rgb)
                for (int c = 0; c < 3; c++) out_rgb[r * 3 + c] = res.rgb[c];
            if (out_aux)
                for (int c = 0; c < 8; c++) out_aux[r * 8 + c] = res.aux[c];
            if (out_nsamp) out_nsamp[r] = res.nsamp;
        }
        free(sv.v);
        free(seg);
        free(order);
    }
}

/* Independent rays with per-block MLPs: each ray sorts the blocks ids from
 * its own origin (as orc_render_rays) and composites them by Eq. 5 with
 * block i's MLP at mlps + i * orc_block_mlp_nparam(L). */
void orc_render_rays_block_mlp(const orc_block *blocks, int32_t nb, const int32_t *ids, int32_t n_ids,
                               const float *o, const float *d, int64_t n_rays, const double *mlps, int32_t L,
                               double *out_rgb, double *out_aux, int32_t *out_nsamp) {
    (void)nb;
    const int32_t n_in = 7 + orc_pe_dim(L);
#pragma omp parallel
    {
        sample_vec sv = {0, 0, 0};
        double *x = (double *)malloc((size_t)n_in * sizeof(double));
        int32_t *order = (int32_t *)malloc((size_t)(n_ids ? n_ids : 1) * sizeof(int32_t));
#pragma omp for schedule(dynamic, 16)
        for (int64_t r = 0; r < n_rays; r++) {
            sort_ids_for_ray(blocks, ids, n_ids, o + 3 * r, order);
            double rgb[3], aux[8];
            int32_t ns;
            render_one_ray_block_mlp(blocks, order, n_ids, o + 3 * r, d + 3 * r, mlps, L, x, &sv, rgb, aux, &ns);
            if (out_rgb)
                for (int c = 0; c < 3; c++) out_rgb[r * 3 + c] = rgb[c];
            if (out_aux)
                for (int c = 0; c < 8; c++) out_aux[r * 8 + c] = aux[c];
            if (out_nsamp) out_nsamp[r] = ns;
        }
        free(sv.v);
        free(x);
        free(order);
    }
}

/* Lattice samples of one ray (for tests): writes up to cap (t, block) pairs
 * of the occupied samples, block by block in `order`; returns the count. */
int64_t orc_ray_samples(const orc_block *blocks, const int32_t *order, int32_t n_order, const float *o,
                        const float *d, double *out_t, int32_t *out_block, double *out_alpha, int64_t cap) {
    sample_vec sv = {0, 0, 0};
    for (int k = 0; k < n_order; k++) block_samples(blocks, order[k], o, d, &sv);
    int64_t n = sv.n;
    for (int64_t i = 0; i < n && i < cap; i++) {
        if (out_t) out_t[i] = sv.v[i].t;
        if (out_block) out_block[i] = sv.v[i].block;
        if (out_alpha) out_alpha[i] = sv.v[i].alpha;
    }
    free(sv.v);
    return n;
}

/* The step (delta of Eq. 1) of every occupied sample of one ray, as
 * orc_ray_samples orders them: the block's lattice spacing, or the
 * recurrence's step in an unbounded block. */
int64_t orc_ray_sample_steps(const orc_block *blocks, const int32_t *order, int32_t n_order, const float *o,
                             const float *d, double *out_delta, int64_t cap) {
    sample_vec sv = {0, 0, 0};
    for (int k = 0; k < n_order; k++) block_samples(blocks, order[k], o, d, &sv);
    int64_t n = sv.n;
    for (int64_t i = 0; i < n && i < cap; i++) out_delta[i] = sv.v[i].delta;
    free(sv.v);
    return n;
}

/* ------------------------------------------------------------------------- */
/* Gradient: reverse mode through MLP, Eq. 12 blend, Eq. 11 accumulation,
 * activations and interpolation taps, for rays rendered block-wise (mode 0).
 * dL_drgb: n_rays x 3.  grad_grid[b]: R^3 x 8 doubles, grad_planes[3b+p]:
 * P^2 x 8 doubles, grad_mlp: 499 doubles; all accumulated into (+=).      */

static void atomic_add(double *p, double v) {
#pragma omp atomic
    *p += v;
}

void orc_render_rays_grad(const orc_block *blocks, int32_t nb, const int32_t *ids, int32_t n_ids,
                          const float *o, const float *d, int64_t n_rays, const double *mlp,
                          const double *dL_drgb, double *const *grad_grid, double *const *grad_planes,
                          double *grad_mlp) {
    (void)nb;
#pragma omp parallel
    {
        sample_vec sv = {0, 0, 0};
        int32_t *order = (int32_t *)malloc((size_t)(n_ids ? n_ids : 1) * sizeof(int32_t));
        int64_t *seg = (int64_t *)malloc((size_t)(n_ids + 1) * sizeof(int64_t));
        double *Ck = (double *)malloc((size_t)(n_ids ? n_ids : 1) * 8 * sizeof(double));
        double *gmlp = (double *)calloc(MLP_NPARAM, sizeof(double));
#pragma omp for schedule(dynamic, 16)
        for (int64_t r = 0; r < n_rays; r++) {
            const float *of = o + 3 * r, *df = d + 3 * r;
            sort_ids_for_ray(blocks, ids, n_ids, of, order);
            sv.n = 0;
            seg[0] = 0;
            for (int k = 0; k < n_ids; k++) {
                block_samples(blocks, order[k], of, df, &sv);
                seg[k + 1] = sv.n;
            }
            /* forward, Eq. 11 per block (running product form), Eq. 12 blend */
            double Cd[3] = {0, 0, 0}, F[4] = {0, 0, 0, 0}, B = 1.0;
            for (int k = 0; k < n_ids; k++) {
                double *ck = Ck + 8 * k; /* C^k (3), F^k (4), alpha^k */
                for (int c = 0; c < 8; c++) ck[c] = 0.0;
                double T = 1.0;
                for (int64_t i = seg[k]; i < seg[k + 1]; i++) {
                    const double w = T * sv.v[i].alpha;
                    for (int c = 0; c < 3; c++) ck[c] += w * sv.v[i].c[c];
                    for (int c = 0; c < 4; c++) ck[3 + c] += w * sv.v[i].s[c];
                    ck[7] += w;
                    T *= 1.0 - sv.v[i].alpha;
                }
                for (int c = 0; c < 3; c++) Cd[c] += B * ck[c];
                for (int c = 0; c < 4; c++) F[c] += B * ck[3 + c];
                B *= 1.0 - ck[7];
            }
            /* MLP backward */
            const double *g = dL_drgb + 3 * r;
            double gC[3] = {g[0], g[1], g[2]}, gF[4] = {0, 0, 0, 0};
            {
                double x[MLP_IN] = {Cd[0], Cd[1], Cd[2], F[0], F[1], F[2], F[3], df[0], df[1], df[2]};
                mlp_trace tr;
                mlp_forward(mlp, x, &tr);
                double dz3[MLP_OUT], dh2[MLP_HID], dz2[MLP_HID], dh1[MLP_HID], dz1[MLP_HID];
                for (int j = 0; j < MLP_OUT; j++) dz3[j] = g[j] * tr.o[j] * (1.0 - tr.o[j]);
                for (int i = 0; i < MLP_HID; i++) {
                    dh2[i] = 0.0;
                    for (int j = 0; j < MLP_OUT; j++) {
                        gmlp[OFF_W3 + i * MLP_OUT + j] += tr.h2[i] * dz3[j];
                        dh2[i] += mlp[OFF_W3 + i * MLP_OUT + j] * dz3[j];
                    }
                }
                for (int j = 0; j < MLP_OUT; j++) gmlp[OFF_B3 + j] += dz3[j];
                for (int j = 0; j < MLP_HID; j++) dz2[j] = tr.z2[j] > 0.0 ? dh2[j] : 0.0;
                for (int i = 0; i < MLP_HID; i++) {
                    dh1[i] = 0.0;
                    for (int j = 0; j < MLP_HID; j++) {
                        gmlp[OFF_W2 + i * MLP_HID + j] += tr.h1[i] * dz2[j];
                        dh1[i] += mlp[OFF_W2 + i * MLP_HID + j] * dz2[j];
                    }
                }
                for (int j = 0; j < MLP_HID; j++) gmlp[OFF_B2 + j] += dz2[j];
                for (int j = 0; j < MLP_HID; j++) dz1[j] = tr.z1[j] > 0.0 ? dh1[j] : 0.0;
                for (int i = 0; i < MLP_IN; i++) {
                    double dx = 0.0;
                    for (int j = 0; j < MLP_HID; j++) {
                        gmlp[OFF_W1 + i * MLP_HID + j] += x[i] * dz1[j];
                        dx += mlp[OFF_W1 + i * MLP_HID + j] * dz1[j];
                    }
                    if (i < 3) gC[i] += dx;
                    else if (i < 7) gF[i - 3] += dx;
                }
                for (int j = 0; j < MLP_HID; j++) gmlp[OFF_B1 + j] += dz1[j];
            }
            /* Eq. 12 backward: B_1 = 1, B_{k+1} = B_k (1 - alpha^k) */
            double gBnext = 0.0;
            double *Bk = (double *)malloc((size_t)(n_ids + 1) * sizeof(double));
            Bk[0] = 1.0;
            for (int k = 0; k < n_ids; k++) Bk[k + 1] = Bk[k] * (1.0 - Ck[8 * k + 7]);
            for (int k = n_ids - 1; k >= 0; k--) {
                const double *ck = Ck + 8 * k;
                const double gA = -gBnext * Bk[k];
                double gB = gBnext * (1.0 - ck[7]);
                for (int c = 0; c < 3; c++) gB += gC[c] * ck[c];
                for (int c = 0; c < 4; c++) gB += gF[c] * ck[3 + c];
                gBnext = gB;
                double gCk[3], gFk[4];
                for (int c = 0; c < 3; c++) gCk[c] = Bk[k] * gC[c];
                for (int c = 0; c < 4; c++) gFk[c] = Bk[k] * gF[c];
                /* Eq. 11 backward: w_i = T_i alpha_i, T_{i+1} = T_i (1 - alpha_i) */
                const int64_t n = seg[k + 1] - seg[k];
                if (n == 0) continue;
                double *Ti = (double *)malloc((size_t)n * sizeof(double));
                double T = 1.0;
                for (int64_t i = 0; i < n; i++) {
                    Ti[i] = T;
                    T *= 1.0 - sv.v[seg[k] + i].alpha;
                }
                double U = 0.0; /* sum_{j>i} gw_j w_j / T_{i+1} */
                for (int64_t i = n - 1; i >= 0; i--) {
                    const sample *s = &sv.v[seg[k] + i];
                    const double w = Ti[i] * s->alpha;
                    double gw = gA;
                    for (int c = 0; c < 3; c++) gw += gCk[c] * s->c[c];
                    for (int c = 0; c < 4; c++) gw += gFk[c] * s->s[c];
                    const double galpha = Ti[i] * (gw - U);
                    U = gw * s->alpha + (1.0 - s->alpha) * U;
                    double gf[NCH];
                    /* alpha = 1 - exp(-exp(f0) delta): d alpha / d f0 = sigma delta (1 - alpha) */
                    gf[0] = galpha * s->sigma * s->delta * (1.0 - s->alpha);
                    for (int c = 0; c < 3; c++) gf[1 + c] = w * gCk[c] * s->c[c] * (1.0 - s->c[c]);
                    for (int c = 0; c < 4; c++) gf[4 + c] = w * gFk[c] * s->s[c] * (1.0 - s->s[c]);
                    const int32_t bi = s->block;
                    for (int q = 0; q < 8; q++)
                        for (int c = 0; c < NCH; c++)
                            atomic_add(&grad_grid[bi][s->tp.gidx[q] + c], s->tp.gw[q] * gf[c]);
                    for (int pl = 0; pl < 3; pl++)
                        for (int q = 0; q < 4; q++)
                            for (int c = 0; c < NCH; c++)
                                atomic_add(&grad_planes[3 * bi + pl][s->tp.pidx[pl][q] + c],
                                           s->tp.pw[pl][q] * gf[c]);
                }
                free(Ti);
            }
            free(Bk);
        }
        for (int i = 0; i < MLP_NPARAM; i++) atomic_add(&grad_mlp[i], gmlp[i]);
        free(sv.v);
        free(order);
        free(seg);
        free(Ck);
        free(gmlp);
    }
}

/* ------------------------------------------------------------------------- */
/* Gradient of the per-block form (Eq. 5 with Eq. 3 per block) for rays:
 * C = sum_k B_k (C^k + Phi^k(C^k, F^k, PE(d))), B_{k+1} = B_k (1 - alpha^k),
 * over the blocks with occupied samples.  Reverse mode: with u = B_k dL/dC,
 * block k's MLP receives u (its weights' gradient, and dL/dC^k = u + J_C^T u,
 * dL/dF^k = J_F^T u); dL/dB_k = dL/dC . (C^k + Phi^k) + dL/dB_{k+1} (1 -
 * alpha^k) and dL/dalpha^k = -dL/dB_{k+1} B_k; inside the block the Eq. 11
 * backward of the global form.  grad_mlps: nb x orc_block_mlp_nparam(L)
 * doubles, accumulated (+=) like the feature gradients. */

/* Phi of an n_in-input MLP and its reverse mode for the upstream u (3):
 * adds u's gradient of every weight to gw and writes dPhi/dx^T u to gx. */
static void mlp_n_backward(const double *w, int32_t n_in, const double *x, const double u[MLP_OUT],
                           double phi[MLP_OUT], double *gx, double *gw) {
    const double *W1 = w, *b1 = W1 + n_in * MLP_HID, *W2 = b1 + MLP_HID, *b2 = W2 + MLP_HID * MLP_HID;
    const double *W3 = b2 + MLP_HID;
    const double *b3 = W3 + MLP_HID * MLP_OUT;
    double *gW1 = gw, *gb1 = gW1 + n_in * MLP_HID, *gW2 = gb1 + MLP_HID, *gb2 = gW2 + MLP_HID * MLP_HID;
    double *gW3 = gb2 + MLP_HID, *gb3 = gW3 + MLP_HID * MLP_OUT;
    double z1[MLP_HID], h1[MLP_HID], z2[MLP_HID], h2[MLP_HID];
    for (int j = 0; j < MLP_HID; j++) {
        double a = b1[j];
        for (int i = 0; i < n_in; i++) a += x[i] * W1[i * MLP_HID + j];
        z1[j] = a;
        h1[j] = a > 0.0 ? a : 0.0;
    }
    for (int j = 0; j < MLP_HID; j++) {
        double a = b2[j];
        for (int i = 0; i < MLP_HID; i++) a += h1[i] * W2[i * MLP_HID + j];
        z2[j] = a;
        h2[j] = a > 0.0 ? a : 0.0;
    }
    double dz3[MLP_OUT], dh2[MLP_HID], dz2[MLP_HID], dh1[MLP_HID], dz1[MLP_HID];
    for (int j = 0; j < MLP_OUT; j++) {
        double a = b3[j];
        for (int i = 0; i < MLP_HID; i++) a += h2[i] * W3[i * MLP_OUT + j];
        phi[j] = sigmoid(a);
        dz3[j] = u[j] * phi[j] * (1.0 - phi[j]);
        gb3[j] += dz3[j];
    }
    for (int i = 0; i < MLP_HID; i++) {
        dh2[i] = 0.0;
        for (int j = 0; j < MLP_OUT; j++) {
            gW3[i * MLP_OUT + j] += h2[i] * dz3[j];
            dh2[i] += W3[i * MLP_OUT + j] * dz3[j];
        }
    }
    for (int j = 0; j < MLP_HID; j++) {
        dz2[j] = z2[j] > 0.0 ? dh2[j] : 0.0;
        gb2[j] += dz2[j];
    }
    for (int i = 0; i < MLP_HID; i++) {
        dh1[i] = 0.0;
        for (int j = 0; j < MLP_HID; j++) {
            gW2[i * MLP_HID + j] += h1[i] * dz2[j];
            dh1[i] += W2[i * MLP_HID + j] * dz2[j];
        }
    }
    for (int j = 0; j < MLP_HID; j++) {
        dz1[j] = z1[j] > 0.0 ? dh1[j] : 0.0;
        gb1[j] += dz1[j];
    }
    for (int i = 0; i < n_in; i++) {
        double dx = 0.0;
        for (int j = 0; j < MLP_HID; j++) {
            gW1[i * MLP_HID + j] += x[i] * dz1[j];
            dx += W1[i * MLP_HID + j] * dz1[j];
        }
        gx[i] = dx;
    }
}

/* Scatter one sample's feature gradient gf (8 channels) through its taps. */
static void scatter_feature_grad(const sample *s, const double gf[NCH], double *const *grad_grid,
                                 double *const *grad_planes) {
    const int32_t bi = s->block;
    for (int q = 0; q < 8; q++)
        for (int c = 0; c < NCH; c++) atomic_add(&grad_grid[bi][s->tp.gidx[q] + c], s->tp.gw[q] * gf[c]);
    for (int pl = 0; pl < 3; pl++)
        for (int q = 0; q < 4; q++)
            for (int c = 0; c < NCH; c++)
                atomic_add(&grad_planes[3 * bi + pl][s->tp.pidx[pl][q] + c], s->tp.pw[pl][q] * gf[c]);
}

void orc_render_rays_block_mlp_grad(const orc_block *blocks, int32_t nb, const int32_t *ids, int32_t n_ids,
                                    const float *o, const float *d, int64_t n_rays, const double *mlps, int32_t L,
                                    const double *dL_drgb, double *const *grad_grid, double *const *grad_planes,
                                    double *grad_mlps) {
    const int32_t n_in = 7 + orc_pe_dim(L), np = orc_block_mlp_nparam(L);
#pragma omp parallel
    {
        sample_vec sv = {0, 0, 0};
        int32_t *order = (int32_t *)malloc((size_t)(n_ids ? n_ids : 1) * sizeof(int32_t));
        int64_t *seg = (int64_t *)malloc((size_t)(n_ids + 1) * sizeof(int64_t));
        double *Ck = (double *)malloc((size_t)(n_ids ? n_ids : 1) * 8 * sizeof(double));
        double *Bk = (double *)malloc((size_t)(n_ids + 1) * sizeof(double));
        double *x = (double *)malloc((size_t)n_in * sizeof(double));
        double *gx = (double *)malloc((size_t)n_in * sizeof(double));
        double *gw = (double *)calloc((size_t)nb * (size_t)np, sizeof(double)); /* this thread's MLP gradients */
        double *Tin = NULL; /* in-block transmittance before each sample */
        int64_t tcap = 0;
#pragma omp for schedule(dynamic, 16)
        for (int64_t r = 0; r < n_rays; r++) {
            const float *of = o + 3 * r, *df = d + 3 * r;
            const double dd[3] = {df[0], df[1], df[2]};
            sort_ids_for_ray(blocks, ids, n_ids, of, order);
            sv.n = 0;
            seg[0] = 0;
            for (int k = 0; k < n_ids; k++) {
                block_samples(blocks, order[k], of, df, &sv);
                seg[k + 1] = sv.n;
            }
            if (sv.n > tcap) {
                tcap = sv.n;
                Tin = (double *)realloc(Tin, (size_t)tcap * sizeof(double));
            }
            /* forward: Eq. 11 per block; B_k over the blocks with samples */
            Bk[0] = 1.0;
            for (int k = 0; k < n_ids; k++) {
                double *ck = Ck + 8 * k; /* C^k (3), F^k (4), alpha^k */
                for (int c = 0; c < 8; c++) ck[c] = 0.0;
                double T = 1.0;
                for (int64_t i = seg[k]; i < seg[k + 1]; i++) {
                    Tin[i] = T;
                    const double w = T * sv.v[i].alpha;
                    for (int c = 0; c < 3; c++) ck[c] += w * sv.v[i].c[c];
                    for (int c = 0; c < 4; c++) ck[3 + c] += w * sv.v[i].s[c];
                    ck[7] += w;
                    T *= 1.0 - sv.v[i].alpha;
                }
                Bk[k + 1] = Bk[k] * (1.0 - ck[7]);
            }
            /* reverse over the blocks */
            const double *g = dL_drgb + 3 * r;
            double gBnext = 0.0;
            for (int k = n_ids - 1; k >= 0; k--) {
                const int64_t n = seg[k + 1] - seg[k];
                if (n == 0) continue; /* a block without occupied samples takes no part */
                const double *ck = Ck + 8 * k;
                for (int c = 0; c < 7; c++) x[c] = ck[c];
                orc_pe(dd, L, x + 7);
                const double u[MLP_OUT] = {Bk[k] * g[0], Bk[k] * g[1], Bk[k] * g[2]};
                double phi[MLP_OUT];
                mlp_n_backward(mlps + (int64_t)order[k] * np, n_in, x, u, phi, gx, gw + (int64_t)order[k] * np);
                const double gA = -gBnext * Bk[k];
                double gB = gBnext * (1.0 - ck[7]);
                for (int c = 0; c < 3; c++) gB += g[c] * (ck[c] + phi[c]);
                gBnext = gB;
                double gCk[3], gFk[4];
                for (int c = 0; c < 3; c++) gCk[c] = u[c] + gx[c];
                for (int c = 0; c < 4; c++) gFk[c] = gx[3 + c];
                /* Eq. 11 backward, as in the global form */
                double U = 0.0;
                for (int64_t i = n - 1; i >= 0; i--) {
                    const sample *s = &sv.v[seg[k] + i];
                    const double T = Tin[seg[k] + i];
                    const double w = T * s->alpha;
                    double gw_i = gA;
                    for (int c = 0; c < 3; c++) gw_i += gCk[c] * s->c[c];
                    for (int c = 0; c < 4; c++) gw_i += gFk[c] * s->s[c];
                    const double galpha = T * (gw_i - U);
                    U = gw_i * s->alpha + (1.0 - s->alpha) * U;
                    double gf[NCH];
                    gf[0] = galpha * s->sigma * s->delta * (1.0 - s->alpha);
                    for (int c = 0; c < 3; c++) gf[1 + c] = w * gCk[c] * s->c[c] * (1.0 - s->c[c]);
                    for (int c = 0; c < 4; c++) gf[4 + c] = w * gFk[c] * s->s[c] * (1.0 - s->s[c]);
                    scatter_feature_grad(s, gf, grad_grid, grad_planes);
                }
            }
        }
        for (int64_t i = 0; i < (int64_t)nb * np; i++)
            if (gw[i] != 0.0) atomic_add(&grad_mlps[i], gw[i]);
        free(sv.v);
        free(order);
        free(seg);
        free(Ck);
        free(Bk);
        free(x);
        free(gx);
        free(gw);
        free(Tin);
    }
}

/* ------------------------------------------------------------------------- */
/* Training-stage regularisers of Sec. 4.3 on the baked representation, with
 * their gradients (accumulated into the same arrays as above).
 *
 * Sparsity (Eq. 7): the mean over given points p of |alpha(p)|, alpha(p) =
 * 1 - exp(-sigma(p) delta_b) with sigma from the block that contains p
 * (Eq. 4 membership on the FP32 point, the extended region of an unbounded
 * block; the first such block in ids) and that block's lattice spacing
 * delta_b; a point in no block contributes 0.
 * d alpha / d f0 = sigma delta (1 - alpha).
 *
 * Opacity (Eq. 8): for every ray and every block with at least one occupied
 * sample on it, the block opacity alpha^k = 1 - prod_i (1 - alpha_i) (Eq. 11)
 * enters -[a log a + (1 - a) log(1 - a)] with a = alpha^k clamped to
 * [1e-6, 1 - 1e-6]; the loss is the mean over rays of the sum over blocks.
 * d alpha^k / d f0_i = sigma_i delta (1 - alpha^k); the clamp's derivative is
 * 0 outside the interval.  No early termination.
 *
 * Both return weight * loss and add weight * dloss/dparam to the gradients. */

static void scatter_ch0(const sample *s, double g0, double *const *grad_grid, double *const *grad_planes) {
    const int32_t bi = s->block;
    for (int q = 0; q < 8; q++) atomic_add(&grad_grid[bi][s->tp.gidx[q]], s->tp.gw[q] * g0);
    for (int pl = 0; pl < 3; pl++)
        for (int q = 0; q < 4; q++) atomic_add(&grad_planes[3 * bi + pl][s->tp.pidx[pl][q]], s->tp.pw[pl][q] * g0);
}

double orc_sparsity_loss_grad(const orc_block *blocks, int32_t nb, const int32_t *ids, int32_t n_ids,
                              const float *pts, int64_t n_pts, double weight, double *const *grad_grid,
                              double *const *grad_planes) {
    (void)nb;
    double loss = 0.0;
#pragma omp parallel for schedule(static) reduction(+ : loss)
    for (int64_t r = 0; r < n_pts; r++) {
        const float *pf = pts + 3 * r;
        int32_t bi = -1;
        for (int k = 0; k < n_ids && bi < 0; k++) {
            const orc_block *c = &blocks[ids[k]];
            if ((c->unbounded & ORC_CONTRACTED) ? owned_unbounded(c, pf) : inside_block(c, pf)) bi = ids[k];
        }
        if (bi < 0) continue;
        const orc_block *b = &blocks[bi];
        sample s;
        const double p[3] = {pf[0], pf[1], pf[2]};
        if (b->unbounded & ORC_CONTRACTED) {
            double x64[3], u64[3];
            for (int a = 0; a < 3; a++)
                x64[a] = (p[a] - 0.5 * ((double)b->lo[a] + (double)b->hi[a])) / (0.5 * ((double)b->hi[a] - (double)b->lo[a]));
            orc_contract(x64, u64);
            make_taps_u(b, u64, &s.tp);
        } else {
            make_taps(b, p, &s.tp);
        }
        double f[NCH];
        eval_feature(b, &s.tp, f);
        s.block = bi;
        s.delta = (double)block_delta(b);
        s.sigma = exp(f[0]);
        s.alpha = -expm1(-s.sigma * s.delta);
        loss += s.alpha;
        if (grad_grid) scatter_ch0(&s, weight / (double)n_pts * s.sigma * s.delta * (1.0 - s.alpha), grad_grid, grad_planes);
    }
    return weight * loss / (double)(n_pts > 0 ? n_pts : 1);
}

double orc_opacity_loss_grad(const orc_block *blocks, int32_t nb, const int32_t *ids, int32_t n_ids,
                             const float *o, const float *d, int64_t n_rays, double weight,
                             double *const *grad_grid, double *const *grad_planes) {
    (void)nb;
    const double eps = 1e-6;
    double loss = 0.0;
#pragma omp parallel reduction(+ : loss)
    {
        sample_vec sv = {0, 0, 0};
        int32_t *order = (int32_t *)malloc((size_t)(n_ids ? n_ids : 1) * sizeof(int32_t));
#pragma omp for schedule(dynamic, 16)
        for (int64_t r = 0; r < n_rays; r++) {
            sort_ids_for_ray(blocks, ids, n_ids, o + 3 * r, order);
            for (int k = 0; k < n_ids; k++) {
                sv.n = 0;
                const int64_t nk = block_samples(blocks, order[k], o + 3 * r, d + 3 * r, &sv);
                if (nk == 0) continue;
                double T = 1.0;
                for (int64_t i = 0; i < nk; i++) T *= 1.0 - sv.v[i].alpha;
                const double a_raw = 1.0 - T;
                const double a = a_raw < eps ? eps : a_raw > 1.0 - eps ? 1.0 - eps : a_raw;
                loss += -(a * log(a) + (1.0 - a) * log(1.0 - a));
                if (!grad_grid || !(a_raw > eps && a_raw < 1.0 - eps)) continue;
                const double ga = -weight / (double)n_rays * log(a / (1.0 - a)); /* dL / d alpha^k */
                for (int64_t i = 0; i < nk; i++)
                    scatter_ch0(&sv.v[i], ga * sv.v[i].sigma * sv.v[i].delta * T, grad_grid, grad_planes);
            }
        }
        free(sv.v);
        free(order);
    }
    return weight * loss / (double)(n_rays > 0 ? n_rays : 1);
}

/* ------------------------------------------------------------------------- */
/* LOD selection, visibility and depth sorting (Appendix D).                 */

/* Height of the highest occupied part of a block: the top vertex of its
 * highest occupied cell row, in world units; lo_z for an empty block. */
double orc_block_ztop(const orc_block *b) {
    const int Nc = orc_occ_cells(b->R, b->occ_cell);
    int czmax = -1;
    for (int cz = Nc - 1; cz >= 0 && czmax < 0; cz--)
        for (int cy = 0; cy < Nc && czmax < 0; cy++)
            for (int cx = 0; cx < Nc; cx++) {
                int64_t c = ((int64_t)cz * Nc + cy) * Nc + cx;
                if (!b->occ || ((b->occ[c >> 5] >> (c & 31)) & 1u)) {
                    czmax = cz;
                    break;
                }
            }
    if (czmax < 0) return (double)b->lo[2];
    int top = (czmax + 1) * b->occ_cell;
    if (top > b->R - 1) top = b->R - 1;
    return (double)b->lo[2] + ((double)top * ((double)b->hi[2] - (double)b->lo[2])) / (double)(b->R - 1);
}

/* Conservative visibility: the box [lo_x, hi_x] x [lo_y, hi_y] x [lo_z, z_top]
 * is culled when all 8 corners lie strictly outside one of the five planes
 * bounding the view pyramid (apex at the camera, through the image edges). */
static int box_visible(const orc_camera *cam, const double lo[3], const double hi[3]) {
    const double f = focal_length(cam->height, cam->fov_y_deg);
    const double kx = (double)cam->width / (2.0 * f);
    const double ky = (double)cam->height / (2.0 * f);
    const double *m = cam->c2w;
    int out[5] = {1, 1, 1, 1, 1};
    for (int corner = 0; corner < 8; corner++) {
        const double p[3] = {(corner & 1) ? hi[0] : lo[0], (corner & 2) ? hi[1] : lo[1],
                             (corner & 4) ? hi[2] : lo[2]};
        const double q[3] = {p[0] - m[3], p[1] - m[7], p[2] - m[11]};
        /* camera coordinates: R^T q */
        const double xc = (m[0] * q[0] + m[4] * q[1]) + m[8] * q[2];
        const double yc = (m[1] * q[0] + m[5] * q[1]) + m[9] * q[2];
        const double zc = (m[2] * q[0] + m[6] * q[1]) + m[10] * q[2];
        const double depth = -zc;
        const double v[5] = {depth, xc + kx * depth, kx * depth - xc, yc + ky * depth, ky * depth - yc};
        for (int k = 0; k < 5; k++)
            if (v[k] >= 0.0) out[k] = 0;
    }
    for (int k = 0; k < 5; k++)
        if (out[k]) return 0;
    return 1;
}

typedef struct lod_ctx {
    const orc_block *blocks;
    int32_t nb;
    const double *ztop;
    const orc_camera *cam;
    const double *thresh; /* thresh[l-1] for blocks at level l */
    int32_t n_lod;
    int32_t *out;
    int32_t n, cap;
} lod_ctx;

static int lod_visible(const lod_ctx *L, int32_t i) {
    const orc_block *b = &L->blocks[i];
    const double lo[3] = {b->lo[0], b->lo[1], b->lo[2]};
    const double hi[3] = {b->hi[0], b->hi[1], L->ztop[i]};
    return box_visible(L->cam, lo, hi);
}

static double lod_distance(const lod_ctx *L, int32_t i) {
    const orc_block *b = &L->blocks[i];
    const double *m = L->cam->c2w;
    const double dx = 0.5 * ((double)b->lo[0] + (double)b->hi[0]) - m[3];
    const double dy = 0.5 * ((double)b->lo[1] + (double)b->hi[1]) - m[7];
    const double dz = L->ztop[i] - m[11];
    return sqrt((dx * dx + dy * dy) + dz * dz);
}

static void lod_emit(lod_ctx *L, int32_t i) {
    if (L->n < L->cap) L->out[L->n] = i;
    L->n++;
}

/* A visible block at level l > 1 is kept when every visible child (level
 * l-1) is farther than thresh[l-2]; otherwise its visible children are
 * examined in turn.  Level-1 blocks are always kept. */
static void lod_descend(lod_ctx *L, int32_t i) {
    const orc_block *b = &L->blocks[i];
    if (b->level <= 1) {
        lod_emit(L, i);
        return;
    }
    int all_far = 1;
    for (int32_t j = 0; j < L->nb; j++) {
        if (L->blocks[j].parent != i || !lod_visible(L, j)) continue;
        const int32_t lc = L->blocks[j].level;
        const double tau = (lc - 1 < L->n_lod && lc >= 1) ? L->thresh[lc - 1] : 0.0;
        if (!(lod_distance(L, j) > tau)) all_far = 0;
    }
    if (all_far) {
        lod_emit(L, i);
        return;
    }
    for (int32_t j = 0; j < L->nb; j++)
        if (L->blocks[j].parent == i && lod_visible(L, j)) lod_descend(L, j);
}

/* xy distance of the block centre to the camera, squared, in double */
static double sort_key_view(const orc_block *b, const orc_camera *cam) {
    const double dx = 0.5 * ((double)b->lo[0] + (double)b->hi[0]) - cam->c2w[3];
    const double dy = 0.5 * ((double)b->lo[1] + (double)b->hi[1]) - cam->c2w[7];
    return dx * dx + dy * dy;
}

/* Returns the number of selected blocks (written near to far into out_ids
 * when it does not exceed cap). */
int32_t orc_select_lod(const orc_block *blocks, int32_t nb, const orc_camera *cam, const double *lod_thresh,
                       int32_t n_lod, int32_t *out_ids, int32_t cap) {
    double *ztop = (double *)malloc((size_t)(nb ? nb : 1) * sizeof(double));
    int32_t maxlev = 1;
    for (int32_t i = 0; i < nb; i++) {
        ztop[i] = orc_block_ztop(&blocks[i]);
        if (blocks[i].level > maxlev) maxlev = blocks[i].level;
    }
    lod_ctx L = {blocks, nb, ztop, cam, lod_thresh, n_lod, out_ids, 0, cap};
    for (int32_t i = 0; i < nb; i++)
        if (blocks[i].level == maxlev && lod_visible(&L, i)) lod_descend(&L, i);
    int32_t n = L.n;
    if (n <= cap) {
        /* depth sort: xy distance of block centres to the camera, ties by index */
        for (int32_t a = 1; a < n; a++) {
            int32_t id = out_ids[a];
            double k = sort_key_view(&blocks[id], cam);
            int32_t j = a - 1;
            while (j >= 0) {
                double kj = sort_key_view(&blocks[out_ids[j]], cam);
                if (kj > k || (kj == k && out_ids[j] > id)) {
                    out_ids[j + 1] = out_ids[j];
                    j--;
                } else
                    break;
            }
            out_ids[j + 1] = id;
        }
    }
    free(ztop);
    return n;
}

/* Every selected block in depth order without LOD logic (single-level scenes). */
void orc_sort_view(const orc_block *blocks, const int32_t *ids, int32_t n, const orc_camera *cam,
                   int32_t *out) {
    for (int32_t a = 0; a < n; a++) out[a] = ids[a];
    for (int32_t a = 1; a < n; a++) {
        int32_t id = out[a];
        double k = sort_key_view(&blocks[id], cam);
        int32_t j = a - 1;
        while (j >= 0) {
            double kj = sort_key_view(&blocks[out[j]], cam);
            if (kj > k || (kj == k && out[j] > id)) {
                out[j + 1] = out[j];
                j--;
            } else
                break;
        }
        out[j + 1] = id;
    }
}
