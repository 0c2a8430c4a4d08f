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
