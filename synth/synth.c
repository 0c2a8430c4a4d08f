/*
 * synth.c -- seeded synthetic inputs shared by the oracle, the tests and the
 * benchmark.  Nothing here computes any part of the ray-casting method: it
 * only makes volumes (RGBA8 words, 0 = empty voxel) and random numbers.
 *
 * Random numbers come from one counter-based generator, SplitMix64
 * (G. L. Steele, D. Lea, C. H. Flood, "Fast splittable pseudorandom number
 * generators", OOPSLA 2014), applied to a key built from (seed, counters).
 *
 * Build: gcc -O2 -fopenmp -ffp-contract=off -fPIC -shared (no fast-math), so
 * every value is deterministic and independent of the thread count.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

static inline uint64_t sm64(uint64_t x) {
    x += 0x9E3779B97F4A7C15ull;
    x = (x ^ (x >> 30)) * 0xBF58476D1CE4E5B9ull;
    x = (x ^ (x >> 27)) * 0x94D049BB133111EBull;
    return x ^ (x >> 31);
}

/* Hash of (seed, a, b, c, d): SplitMix64 chained over the counters. */
uint64_t sy_hash(uint64_t seed, uint64_t a, uint64_t b, uint64_t c, uint64_t d) {
    uint64_t h = sm64(seed);
    h = sm64(h ^ a);
    h = sm64(h ^ (b + 0x1000000000ull));
    h = sm64(h ^ (c + 0x2000000000ull));
    h = sm64(h ^ (d + 0x3000000000ull));
    return h;
}

/* Uniform double in [0, 1) with 53 random bits. */
static inline double u01(uint64_t h) { return (double)(h >> 11) * 0x1.0p-53; }

double sy_u01(uint64_t seed, uint64_t a, uint64_t b, uint64_t c, uint64_t d) {
    return u01(sy_hash(seed, a, b, c, d));
}

static inline double smooth(double f) { return f * f * (3.0 - 2.0 * f); }

/* ---------------------------------------------------------------------- */
/* Value noise: lattice values u01(hash(seed, i, j, k, octave)) at integer   */
/* lattice points of period `period` voxels, sampled at voxel centres with   */
/* smoothstep-weighted trilinear interpolation.  Result in [0, 1).           */
/* ---------------------------------------------------------------------- */
typedef struct {
    int64_t n;       /* lattice points per axis */
    double* v;       /* n^3 lattice values */
    double period;
} lattice3;

static void lattice3_init(lattice3* L, uint64_t seed, int64_t extent, double period, int octave) {
    L->n = (int64_t)ceil(extent / period) + 2;
    L->period = period;
    L->v = (double*)malloc(sizeof(double) * L->n * L->n * L->n);
    for (int64_t k = 0; k < L->n; k++)
        for (int64_t j = 0; j < L->n; j++)
            for (int64_t i = 0; i < L->n; i++)
                L->v[i + L->n * (j + L->n * k)] = sy_u01(seed, (uint64_t)i, (uint64_t)j, (uint64_t)k, (uint64_t)octave);
}

static inline double lattice3_sample(const lattice3* L, double x, double y, double z) {
    double fx = x / L->period, fy = y / L->period, fz = z / L->period;
    int64_t i = (int64_t)floor(fx), j = (int64_t)floor(fy), k = (int64_t)floor(fz);
    double ax = smooth(fx - i), ay = smooth(fy - j), az = smooth(fz - k);
    const int64_t n = L->n;
    const double* v = L->v;
#define LV(a, b, c) v[(i + (a)) + n * ((j + (b)) + n * (k + (c)))]
    double c00 = LV(0, 0, 0) + ax * (LV(1, 0, 0) - LV(0, 0, 0));
    double c10 = LV(0, 1, 0) + ax * (LV(1, 1, 0) - LV(0, 1, 0));
    double c01 = LV(0, 0, 1) + ax * (LV(1, 0, 1) - LV(0, 0, 1));
    double c11 = LV(0, 1, 1) + ax * (LV(1, 1, 1) - LV(0, 1, 1));
#undef LV
    double c0 = c00 + ay * (c10 - c00);
    double c1 = c01 + ay * (c11 - c01);
    return c0 + az * (c1 - c0);
}

typedef struct {
    int64_t n;
    double* v;
    double period;
} lattice2;

static void lattice2_init(lattice2* L, uint64_t seed, int64_t extent, double period, int octave) {
    L->n = (int64_t)ceil(extent / period) + 2;
    L->period = period;
    L->v = (double*)malloc(sizeof(double) * L->n * L->n);
    for (int64_t j = 0; j < L->n; j++)
        for (int64_t i = 0; i < L->n; i++)
            L->v[i + L->n * j] = sy_u01(seed, (uint64_t)i, (uint64_t)j, 0x2D2D2D, (uint64_t)octave);
}

static inline double lattice2_sample(const lattice2* L, double x, double y) {
    double fx = x / L->period, fy = y / L->period;
    int64_t i = (int64_t)floor(fx), j = (int64_t)floor(fy);
    double ax = smooth(fx - i), ay = smooth(fy - j);
    const int64_t n = L->n;
    const double* v = L->v;
    double c0 = v[i + n * j] + ax * (v[i + 1 + n * j] - v[i + n * j]);
    double c1 = v[i + n * (j + 1)] + ax * (v[i + 1 + n * (j + 1)] - v[i + n * (j + 1)]);
    return c0 + ay * (c1 - c0);
}

/* Single-octave 3D value noise of an N^3 block, sampled at voxel centres.
 * out: N^3 doubles, x fastest. */
void sy_value_noise3(uint64_t seed, int64_t N, double period, double* out) {
    lattice3 L;
    lattice3_init(&L, seed, N, period, 0);
#pragma omp parallel for schedule(static)
    for (int64_t z = 0; z < N; z++)
        for (int64_t y = 0; y < N; y++)
            for (int64_t x = 0; x < N; x++)
                out[x + N * (y + N * z)] = lattice3_sample(&L, x + 0.5, y + 0.5, z + 0.5);
    free(L.v);
}

/* RGBA8 packing: R | G << 8 | B << 16 | A << 24. */
#define RGBA(r, g, b, a) ((uint32_t)(r) | ((uint32_t)(g) << 8) | ((uint32_t)(b) << 16) | ((uint32_t)(a) << 24))

/* ---------------------------------------------------------------------- */
/* Terrain: fBm heightfield (6 octaves) with fBm caves (3 octaves).          */
/* y is up.  Columns are solid below the height; caves carve voxels where    */
/* the cave noise exceeds `cave_tau` and the voxel is 4+ below the surface.  */
/* Materials: top solid voxel of the column = grass, next 3 = dirt, below =  */
/* stone, with two ore colours picked by hash.                               */
/* out: N^3 uint32 (x fastest).  heights_out (optional): N*N doubles.        */
/* ---------------------------------------------------------------------- */
static const uint32_t COL_GRASS = RGBA(60, 160, 60, 255);
static const uint32_t COL_DIRT = RGBA(130, 90, 50, 255);
static const uint32_t COL_STONE = RGBA(120, 120, 124, 255);
static const uint32_t COL_ORE1 = RGBA(210, 170, 40, 255);
static const uint32_t COL_ORE2 = RGBA(50, 100, 210, 255);

void sy_terrain_heights(uint64_t seed, int64_t N, double* h) {
    lattice2 L[6];
    double period = N / 2.0;
    for (int o = 0; o < 6; o++) {
        lattice2_init(&L[o], seed, N, period, o);
        period *= 0.5;
    }
    double norm = 0.0, amp = 1.0;
    for (int o = 0; o < 6; o++) { norm += amp; amp *= 0.5; }
#pragma omp parallel for schedule(static)
    for (int64_t z = 0; z < N; z++)
        for (int64_t x = 0; x < N; x++) {
            double s = 0.0, a = 1.0;
            for (int o = 0; o < 6; o++) {
                s += a * (2.0 * lattice2_sample(&L[o], x + 0.5, z + 0.5) - 1.0);
                a *= 0.5;
            }
            h[x + N * z] = 0.35 * N + 0.3 * N * (s / norm);
        }
    for (int o = 0; o < 6; o++) free(L[o].v);
}

static inline double cave_fbm(const lattice3* C, double x, double y, double z) {
    double s = 0.0, a = 1.0, norm = 0.0;
    for (int o = 0; o < 3; o++) {
        s += a * lattice3_sample(&C[o], x, y, z);
        norm += a;
        a *= 0.5;
    }
    return s / norm;
}

/* Histogram of the cave noise over the voxels that may be carved, on a
 * deterministic subsample (every 4th voxel per axis); returns the value
 * above which `frac` of those voxels lie. */
double sy_terrain_cave_tau(uint64_t seed, int64_t N, const double* h, double frac) {
    lattice3 C[3];
    double period = N / 8.0;
    for (int o = 0; o < 3; o++) { lattice3_init(&C[o], seed ^ 0xCA7Eull, N, period, o); period *= 0.5; }
    enum { NB = 1 << 16 };
    uint64_t* hist = (uint64_t*)calloc(NB, sizeof(uint64_t));
    uint64_t total = 0;
    for (int64_t z = 0; z < N; z += 4)
        for (int64_t x = 0; x < N; x += 4) {
            double top = h[x + N * z] - 4.0;
            for (int64_t y = 0; y < N && (double)y < top; y += 4) {
                double v = cave_fbm(C, x + 0.5, y + 0.5, z + 0.5);
                int64_t b = (int64_t)(v * NB);
                if (b < 0) b = 0;
                if (b >= NB) b = NB - 1;
                hist[b]++;
                total++;
            }
        }
    uint64_t want = (uint64_t)(frac * (double)total), acc = 0;
    double tau = 1.0;
    for (int64_t b = NB - 1; b >= 0; b--) {
        acc += hist[b];
        if (acc >= want) { tau = (double)b / NB; break; }
    }
    free(hist);
    for (int o = 0; o < 3; o++) free(C[o].v);
    return tau;
}

void sy_terrain(uint64_t seed, int64_t N, double cave_tau, const double* h, uint32_t* out) {
    lattice3 C[3];
    double period = N / 8.0;
    for (int o = 0; o < 3; o++) { lattice3_init(&C[o], seed ^ 0xCA7Eull, N, period, o); period *= 0.5; }
#pragma omp parallel for schedule(dynamic, 1)
    for (int64_t z = 0; z < N; z++)
        for (int64_t x = 0; x < N; x++) {
            double hh = h[x + N * z];
            int64_t top = (int64_t)ceil(hh) - 1; /* highest solid y of the column */
            for (int64_t y = 0; y < N; y++) {
                uint32_t w = 0;
                if ((double)y < hh) {
                    int64_t depth = top - y;
                    if (depth == 0) w = COL_GRASS;
                    else if (depth <= 3) w = COL_DIRT;
                    else {
                        uint64_t r = sy_hash(seed ^ 0x0BEull, (uint64_t)x, (uint64_t)y, (uint64_t)z, 7);
                        unsigned m = (unsigned)(r & 1023);
                        w = m < 6 ? COL_ORE1 : (m < 12 ? COL_ORE2 : COL_STONE);
                    }
                    if ((double)y < hh - 4.0 && cave_fbm(C, x + 0.5, y + 0.5, z + 0.5) > cave_tau) w = 0;
                }
                out[x + N * (y + N * z)] = w;
            }
        }
    for (int o = 0; o < 3; o++) free(C[o].v);
}

/* ---------------------------------------------------------------------- */
/* Incoherent rays: origins uniform in [0, N)^3, directions uniform on the   */
/* unit sphere (z ~ U[-1, 1], phi ~ U[0, 2 pi)), tmin = 0, tmax = +inf.      */
/* out: n x 8 floats {ox, oy, oz, tmin, dx, dy, dz, tmax}.                   */
/* ---------------------------------------------------------------------- */
void sy_incoherent_rays(uint64_t seed, int64_t N, int64_t n, float* out) {
    const double TWO_PI = 6.283185307179586476925286766559;
    const float below_n = nextafterf((float)N, 0.0f);
#pragma omp parallel for schedule(static)
    for (int64_t r = 0; r < n; r++) {
        float* o = out + 8 * r;
        for (int a = 0; a < 3; a++) {
            float v = (float)(sy_u01(seed, (uint64_t)r, (uint64_t)a, 0x0A, 0) * (double)N);
            o[a] = v < below_n ? v : below_n;
        }
        double zc = 2.0 * sy_u01(seed, (uint64_t)r, 3, 0x0A, 0) - 1.0;
        double phi = TWO_PI * sy_u01(seed, (uint64_t)r, 4, 0x0A, 0);
        double s = sqrt(fmax(0.0, 1.0 - zc * zc));
        o[3] = 0.0f;
        o[4] = (float)(s * cos(phi));
        o[5] = (float)(s * sin(phi));
        o[6] = (float)zc;
        o[7] = INFINITY;
    }
}

/* Uniform random rays for tiny-grid tests: origins uniform in the box
 * [-m, N + m)^3, directions uniform on the sphere, tmin = 0, tmax = +inf. */
void sy_box_rays(uint64_t seed, double N, double margin, int64_t n, float* out) {
    const double TWO_PI = 6.283185307179586476925286766559;
    for (int64_t r = 0; r < n; r++) {
        float* o = out + 8 * r;
        for (int a = 0; a < 3; a++)
            o[a] = (float)(-margin + sy_u01(seed, (uint64_t)r, (uint64_t)a, 0x0B, 0) * (N + 2.0 * margin));
        double zc = 2.0 * sy_u01(seed, (uint64_t)r, 3, 0x0B, 0) - 1.0;
        double phi = TWO_PI * sy_u01(seed, (uint64_t)r, 4, 0x0B, 0);
        double s = sqrt(fmax(0.0, 1.0 - zc * zc));
        o[3] = 0.0f;
        o[4] = (float)(s * cos(phi));
        o[5] = (float)(s * sin(phi));
        o[6] = (float)zc;
        o[7] = INFINITY;
    }
}

/* ---------------------------------------------------------------------- */
/* Primitive scene (2048^3 workload): seeded spheres, axis-aligned boxes    */
/* and thin walls in world space, plus 64 prototype 64^3 blocks (each a      */
/* small composition of the same primitives) stamped at 64-aligned bricks,  */
/* so identical 64^3 sub-volumes repeat.  Voxel value = palette index of the */
/* last primitive covering the voxel centre (instances override their whole */
/* brick); palette index 0 = empty.  Bricks of 64^3 are produced on demand.  */
/* ---------------------------------------------------------------------- */
enum { PR_SPHERE = 0, PR_BOX = 1 };
typedef struct {
    int type;
    float a[3], b[3]; /* sphere: centre a, radius b[0]; box: [a, b) */
    uint8_t color;
} sy_prim;

typedef struct {
    int64_t n;          /* grid side */
    int64_t nb;         /* bricks per axis (n / 64) */
    int nprim;
    sy_prim* prims;
    int32_t* bin_start; /* nb^3 + 1 */
    int32_t* bin_list;  /* primitive ids per brick, ascending */
    uint8_t* protos;    /* 64 x 64^3 palette indices */
    int32_t* inst;      /* per brick: prototype id or -1 */
    uint32_t palette[256];
    int64_t n_inst;
} sy_scene;

static double rnd(uint64_t seed, uint64_t i, uint64_t k) { return sy_u01(seed, i, k, 0x5C, 0); }

static void prim_bbox(const sy_prim* p, double lo[3], double hi[3]) {
    for (int i = 0; i < 3; i++) {
        if (p->type == PR_SPHERE) { lo[i] = p->a[i] - p->b[0]; hi[i] = p->a[i] + p->b[0]; }
        else { lo[i] = p->a[i]; hi[i] = p->b[i]; }
    }
}

static void make_prim(uint64_t seed, uint64_t i, double extent, double scale, sy_prim* p) {
    double u = rnd(seed, i, 0);
    p->color = (uint8_t)(1 + (sy_hash(seed, i, 99, 0, 0) & 15));
    double c[3];
    for (int k = 0; k < 3; k++) c[k] = rnd(seed, i, 1 + k) * extent;
    if (u < 0.72) { /* sphere, radius log-uniform in [2, 48] * scale */
        p->type = PR_SPHERE;
        double r = 2.0 * exp(rnd(seed, i, 4) * log(24.0)) * scale;
        for (int k = 0; k < 3; k++) p->a[k] = (float)c[k];
        p->b[0] = (float)r; p->b[1] = p->b[2] = 0.0f;
    } else if (u < 0.96) { /* box, edges log-uniform in [2, 96] * scale */
        p->type = PR_BOX;
        for (int k = 0; k < 3; k++) {
            double e = 2.0 * exp(rnd(seed, i, 5 + k) * log(48.0)) * scale;
            p->a[k] = (float)floor(c[k] - e / 2); p->b[k] = (float)floor(c[k] + e / 2) + 1.0f;
        }
    } else { /* thin wall: 1-2 thick on one axis, 128-1024 long on the others */
        p->type = PR_BOX;
        int thin = (int)(sy_hash(seed, i, 98, 0, 0) % 3);
        for (int k = 0; k < 3; k++) {
            double e = k == thin ? 1.0 + (double)(sy_hash(seed, i, 97, k, 0) & 1)
                                 : 128.0 * exp(rnd(seed, i, 8 + k) * log(8.0)) * (scale < 1 ? scale : 1);
            p->a[k] = (float)floor(c[k] - e / 2); p->b[k] = p->a[k] + (float)floor(e);
        }
    }
}

static inline int prim_covers(const sy_prim* p, double x, double y, double z) {
    if (p->type == PR_SPHERE) {
        double dx = x - p->a[0], dy = y - p->a[1], dz = z - p->a[2];
        return dx * dx + dy * dy + dz * dz <= (double)p->b[0] * p->b[0];
    }
    return x >= p->a[0] && x < p->b[0] && y >= p->a[1] && y < p->b[1] && z >= p->a[2] && z < p->b[2];
}

/* Rasterises primitives [ids] over the cube [x0, x0+s)^3 into out (s^3, x fastest). */
static void raster(const sy_prim* prims, const int32_t* ids, int nids, int64_t x0, int64_t y0, int64_t z0, int64_t s,
                   uint8_t* out) {
    for (int q = 0; q < nids; q++) {
        const sy_prim* p = &prims[ids[q]];
        double lo[3], hi[3];
        prim_bbox(p, lo, hi);
        int64_t a[3], b[3];
        const int64_t o[3] = {x0, y0, z0};
        int skip = 0;
        for (int k = 0; k < 3; k++) {
            a[k] = (int64_t)floor(lo[k] - 0.5) - o[k];
            b[k] = (int64_t)ceil(hi[k] + 0.5) - o[k];
            if (a[k] < 0) a[k] = 0;
            if (b[k] > s) b[k] = s;
            if (a[k] >= b[k]) skip = 1;
        }
        if (skip) continue;
        for (int64_t z = a[2]; z < b[2]; z++)
            for (int64_t y = a[1]; y < b[1]; y++)
                for (int64_t x = a[0]; x < b[0]; x++)
                    if (prim_covers(p, x0 + x + 0.5, y0 + y + 0.5, z0 + z + 0.5)) out[x + s * (y + s * z)] = p->color;
    }
}

sy_scene* sy_scene_new(uint64_t seed, int64_t n, int nprim, double scale, int n_proto, int stamps_per_proto) {
    sy_scene* S = (sy_scene*)calloc(1, sizeof(sy_scene));
    S->n = n;
    S->nb = n / 64;
    S->nprim = nprim;
    S->prims = (sy_prim*)malloc(sizeof(sy_prim) * (nprim > 0 ? nprim : 1));
    for (int i = 0; i < nprim; i++) make_prim(seed, (uint64_t)i, (double)n, scale, &S->prims[i]);
    /* palette: 16 colours */
    S->palette[0] = 0;
    for (int c = 1; c < 256; c++) {
        uint64_t h = sy_hash(seed ^ 0xC0102ull, (uint64_t)c, 0, 0, 0);
        S->palette[c] = (uint32_t)(h & 0x00FFFFFFu) | 0xFF000000u;
    }
    /* bins: primitive ids per 64^3 brick */
    const int64_t nb = S->nb, nbins = nb * nb * nb;
    int32_t* cnt = (int32_t*)calloc((size_t)nbins, sizeof(int32_t));
    for (int pass = 0; pass < 2; pass++) {
        if (pass == 1) {
            S->bin_start = (int32_t*)malloc(sizeof(int32_t) * (size_t)(nbins + 1));
            S->bin_start[0] = 0;
            for (int64_t b = 0; b < nbins; b++) S->bin_start[b + 1] = S->bin_start[b] + cnt[b];
            S->bin_list = (int32_t*)malloc(sizeof(int32_t) * (size_t)(S->bin_start[nbins] + 1));
            memset(cnt, 0, sizeof(int32_t) * (size_t)nbins);
        }
        for (int i = 0; i < nprim; i++) {
            double lo[3], hi[3];
            prim_bbox(&S->prims[i], lo, hi);
            int64_t a[3], b[3];
            for (int k = 0; k < 3; k++) {
                a[k] = (int64_t)floor((lo[k] - 1.0) / 64.0);
                b[k] = (int64_t)floor((hi[k] + 1.0) / 64.0);
                if (a[k] < 0) a[k] = 0;
                if (b[k] > nb - 1) b[k] = nb - 1;
            }
            for (int64_t z = a[2]; z <= b[2]; z++)
                for (int64_t y = a[1]; y <= b[1]; y++)
                    for (int64_t x = a[0]; x <= b[0]; x++) {
                        int64_t bi = x + nb * (y + nb * z);
                        if (pass == 1) S->bin_list[S->bin_start[bi] + cnt[bi]] = i;
                        cnt[bi]++;
                    }
        }
    }
    free(cnt);
    /* prototypes: each 6 primitives inside a 64^3 block */
    S->protos = (uint8_t*)calloc((size_t)n_proto * 64 * 64 * 64 + 1, 1);
    for (int pi = 0; pi < n_proto; pi++) {
        sy_prim pp[6];
        int32_t ids[6];
        for (int q = 0; q < 6; q++) {
            make_prim(seed ^ 0x9A0707ull, (uint64_t)(pi * 6 + q), 64.0, 0.5, &pp[q]);
            ids[q] = q;
        }
        raster(pp, ids, 6, 0, 0, 0, 64, S->protos + (size_t)pi * 64 * 64 * 64);
    }
    /* instances: stamps_per_proto stamps of each prototype at seeded bricks */
    S->inst = (int32_t*)malloc(sizeof(int32_t) * (size_t)nbins);
    for (int64_t b = 0; b < nbins; b++) S->inst[b] = -1;
    S->n_inst = 0;
    for (int pi = 0; pi < n_proto; pi++)
        for (int k = 0; k < stamps_per_proto; k++) {
            uint64_t h = sy_hash(seed ^ 0x57A3Bull, (uint64_t)pi, (uint64_t)k, 0, 0);
            int64_t bi = (int64_t)(h % (uint64_t)nbins);
            if (S->inst[bi] < 0) S->n_inst++;
            S->inst[bi] = pi;
        }
    return S;
}

void sy_scene_free(sy_scene* S) {
    if (!S) return;
    free(S->prims); free(S->bin_start); free(S->bin_list); free(S->protos); free(S->inst);
    free(S);
}

const uint32_t* sy_scene_palette(const sy_scene* S) { return S->palette; }
int64_t sy_scene_instances(const sy_scene* S) { return S->n_inst; }

/* Palette indices of the 64^3 brick (bx, by, bz). */
static void scene_brick_u8(const sy_scene* S, int64_t bx, int64_t by, int64_t bz, uint8_t* out) {
    const int64_t bi = bx + S->nb * (by + S->nb * bz);
    if (S->inst[bi] >= 0) {
        memcpy(out, S->protos + (size_t)S->inst[bi] * 64 * 64 * 64, 64 * 64 * 64);
        return;
    }
    memset(out, 0, 64 * 64 * 64);
    raster(S->prims, S->bin_list + S->bin_start[bi], S->bin_start[bi + 1] - S->bin_start[bi], bx * 64, by * 64,
           bz * 64, 64, out);
}

/* vx_fill_brick_fn-compatible callback: RGBA words of a cube (side 2^l2 <= 64,
 * corner a multiple of the side), user = the scene. */
int sy_scene_fill_brick(void* user, uint32_t x0, uint32_t y0, uint32_t z0, uint32_t l2, uint32_t* out) {
    const sy_scene* S = (const sy_scene*)user;
    const int64_t s = (int64_t)1 << l2;
    if (s > 64) {
        for (int64_t z = 0; z < s; z += 64)
            for (int64_t y = 0; y < s; y += 64)
                for (int64_t x = 0; x < s; x += 64) {
                    uint32_t* tmp = (uint32_t*)malloc(sizeof(uint32_t) * 64 * 64 * 64);
                    sy_scene_fill_brick(user, x0 + (uint32_t)x, y0 + (uint32_t)y, z0 + (uint32_t)z, 6, tmp);
                    for (int64_t zz = 0; zz < 64; zz++)
                        for (int64_t yy = 0; yy < 64; yy++)
                            memcpy(out + (x + s * ((y + yy) + s * (z + zz))), tmp + 64 * (yy + 64 * zz), 64 * 4);
                    free(tmp);
                }
        return 0;
    }
    uint8_t* b = (uint8_t*)malloc(64 * 64 * 64);
    const int64_t bx = x0 / 64, by = y0 / 64, bz = z0 / 64;
    scene_brick_u8(S, bx, by, bz, b);
    const int64_t ox = x0 % 64, oy = y0 % 64, oz = z0 % 64;
    for (int64_t z = 0; z < s; z++)
        for (int64_t y = 0; y < s; y++)
            for (int64_t x = 0; x < s; x++)
                out[x + s * (y + s * z)] = S->palette[b[(ox + x) + 64 * ((oy + y) + 64 * (oz + z))]];
    free(b);
    return 0;
}

/* vx_block_empty_fn-compatible: 1 only when no primitive or instance can
 * touch the cube (side >= 64). */
int sy_scene_block_empty(void* user, uint32_t x0, uint32_t y0, uint32_t z0, uint32_t l2) {
    const sy_scene* S = (const sy_scene*)user;
    if (l2 < 6) return 0;
    const int64_t k = (int64_t)1 << (l2 - 6);
    for (int64_t bz = z0 / 64; bz < z0 / 64 + k; bz++)
        for (int64_t by = y0 / 64; by < y0 / 64 + k; by++)
            for (int64_t bx = x0 / 64; bx < x0 / 64 + k; bx++) {
                const int64_t bi = bx + S->nb * (by + S->nb * bz);
                if (S->inst[bi] >= 0 || S->bin_start[bi + 1] > S->bin_start[bi]) return 0;
            }
    return 1;
}

/* Whole grid as palette indices (n^3 bytes, x fastest). Returns occupied count. */
int64_t sy_scene_render_u8(const sy_scene* S, uint8_t* grid) {
    const int64_t nb = S->nb, n = S->n;
    int64_t occ = 0;
#pragma omp parallel for schedule(dynamic, 1) reduction(+ : occ)
    for (int64_t bi = 0; bi < nb * nb * nb; bi++) {
        uint8_t* b = (uint8_t*)malloc(64 * 64 * 64);
        const int64_t bx = bi % nb, by = (bi / nb) % nb, bz = bi / (nb * nb);
        scene_brick_u8(S, bx, by, bz, b);
        for (int64_t z = 0; z < 64; z++)
            for (int64_t y = 0; y < 64; y++) {
                memcpy(grid + (bx * 64) + n * ((by * 64 + y) + n * (bz * 64 + z)), b + 64 * (y + 64 * z), 64);
                for (int x = 0; x < 64; x++) occ += b[x + 64 * (y + 64 * z)] != 0;
            }
        free(b);
    }
    return occ;
}
