/*
 * oracle.c -- plain, slow, FP64 CPU oracle for first-hit ray casting through
 * a voxel volume.
 *
 * TEST INFRASTRUCTURE ONLY.  Only the tests, the smoke check and the
 * benchmark's CPU-baseline leg load this library.  It shares no code, header,
 * table or helper with the CUDA path and includes nothing from it.
 *
 * What it computes
 * ----------------
 * A voxel holds a 32-bit RGBA word and is empty iff all 32 bits are 0
 * (Sec. 3).  The hybrid formats of Sec. 3.1-3.3 are lossless re-encodings of
 * such a grid, and the intersection functions of Sec. 4.2 return the first
 * non-empty voxel hit along the ray, visiting sub-volumes in hit-time order
 * (Fig. 4, ordered_hit_children).  So the answer every format must give is
 * the first occupied voxel along the ray in the uncompressed grid, found here
 * with the Amanatides-Woo stepping that Sec. 2 describes: from the voxel
 * holding the ray, repeatedly step to the neighbour across the nearest voxel
 * boundary.
 *
 * Conventions (the paper renders images and fixes none of these; each is a
 * stated reading):
 *   - world units are voxels; the grid covers [0,nx) x [0,ny) x [0,nz);
 *   - a ray is {o, tmin, d, tmax} in float32, widened exactly to double;
 *     points are o + t d for t in [tmin, tmax];
 *   - entry into the box: t_enter = max(tmin, largest slab entry), the entry
 *     axis is the lowest axis attaining the largest slab entry, and is used
 *     only when that entry is > tmin; t_exit = min(tmax, smallest slab exit);
 *     MISS when t_enter >= t_exit; an axis with d = 0 needs 0 <= o < n;
 *   - start voxel: on the entry axis the first layer (0 if d > 0, else n-1);
 *     on other axes floor(p) of p = o + t_enter d, except p integral with
 *     d < 0 gives p - 1; clamped to the grid;
 *   - each boundary crossing is recomputed in closed form from the integer
 *     plane, ((v + (d > 0)) - o) / d, never accumulated; ties in crossing
 *     time step the lowest axis first;
 *   - the hit t is the entry t of the hit voxel (t_enter for the first
 *     voxel); the face is 1 + 2 axis + (d_axis < 0) of the last step (the
 *     entry axis for the first voxel), 0 when the ray starts inside;
 *   - a ray with a NaN component or a non-finite tmin is INVALID.
 *
 * The file also holds: the near-tie classifier, a brute-force slab checker
 * over every voxel box (tiny grids), an FP64 pinhole ray generator, and a
 * decoder of the paper's word-buffer layout (Sec. 3.3, Fig. 3) back into a
 * dense grid, which also checks every distance a DF level stores.
 *
 * Compiled with -ffp-contract=off and no fast-math: every FP64 expression
 * below is evaluated with one IEEE rounding per operation, in source order.
 */
#include <math.h>
#include <pthread.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

/* ------------------------------------------------------------------------ */
/* Grid access                                                               */
/* ------------------------------------------------------------------------ */
typedef struct {
    const uint32_t* g32; /* dense RGBA words, x fastest; or NULL */
    const uint8_t* g8;   /* dense palette indices, x fastest; or NULL */
    const uint32_t* pal; /* 256-entry palette for g8 (pal[0] must be 0) */
    int64_t n[3];
} grid_t;

static inline uint32_t gval(const grid_t* G, const int64_t v[3]) {
    int64_t i = v[0] + G->n[0] * (v[1] + G->n[1] * v[2]);
    return G->g32 ? G->g32[i] : G->pal[G->g8[i]];
}

static inline int64_t glin(const grid_t* G, const int64_t v[3]) {
    return v[0] + G->n[0] * (v[1] + G->n[1] * v[2]);
}

/* ------------------------------------------------------------------------ */
/* Rays                                                                      */
/* ------------------------------------------------------------------------ */
typedef struct {
    double o[3], d[3], tmin, tmax;
} ray64;

/* Widen a float32 ray exactly; returns 0 for an INVALID ray. */
static int load_ray(const float* r, ray64* R) {
    for (int i = 0; i < 8; i++)
        if (isnan(r[i])) return 0;
    if (isinf(r[3])) return 0;
    R->o[0] = r[0]; R->o[1] = r[1]; R->o[2] = r[2];
    R->tmin = r[3];
    R->d[0] = r[4]; R->d[1] = r[5]; R->d[2] = r[6];
    R->tmax = r[7];
    return 1;
}

typedef struct {
    double t;
    uint32_t rgba;
    int32_t x, y, z;
    int32_t face;
    int32_t status; /* 0 miss, 1 hit, 2 invalid */
    int32_t pad;
} or_hit;

enum { ST_MISS = 0, ST_HIT = 1, ST_INVALID = 2 };

/* Slab test against the whole box.  Returns 0 when an axis with d = 0 lies
 * outside the box (certain miss); otherwise fills t_enter, t_exit and the
 * entry axis (-1 when the ray starts at tmin inside the box) and returns 1;
 * the caller still checks t_enter < t_exit. */
static int root_slab(const grid_t* G, const ray64* R, double* te, double* tx, int* eaxis) {
    double best = -INFINITY, texit = R->tmax;
    int bax = -1;
    for (int i = 0; i < 3; i++) {
        double n = (double)G->n[i];
        if (R->d[i] == 0.0) {
            if (!(R->o[i] >= 0.0 && R->o[i] < n)) return 0;
            continue;
        }
        double lo = R->d[i] > 0.0 ? 0.0 : n;
        double hi = R->d[i] > 0.0 ? n : 0.0;
        double t0 = (lo - R->o[i]) / R->d[i];
        double t1 = (hi - R->o[i]) / R->d[i];
        if (t0 > best) { best = t0; bax = i; }
        if (t1 < texit) texit = t1;
    }
    if (bax >= 0 && best > R->tmin) { *te = best; *eaxis = bax; }
    else { *te = R->tmin; *eaxis = -1; }
    *tx = texit;
    return 1;
}

static void start_voxel(const grid_t* G, const ray64* R, double te, int e, int64_t v[3]) {
    for (int i = 0; i < 3; i++) {
        int64_t vi;
        if (i == e) {
            vi = R->d[i] > 0.0 ? 0 : G->n[i] - 1;
        } else {
            double p = R->o[i] + te * R->d[i];
            double f = floor(p);
            if (f < -1.0) f = -1.0;
            if (f > (double)G->n[i]) f = (double)G->n[i];
            vi = (int64_t)f;
            if (p == f && R->d[i] < 0.0) vi -= 1;
        }
        if (vi < 0) vi = 0;
        if (vi > G->n[i] - 1) vi = G->n[i] - 1;
        v[i] = vi;
    }
}

static inline double t_cross(const ray64* R, int i, int64_t v) {
    /* Time at which the ray leaves cell v on axis i (closed form). */
    if (R->d[i] == 0.0) return INFINITY;
    double plane = (double)(v + (R->d[i] > 0.0 ? 1 : 0));
    return (plane - R->o[i]) / R->d[i];
}

static inline int face_of(const ray64* R, int a) { return 1 + 2 * a + (R->d[a] < 0.0 ? 1 : 0); }

/* The exact-order FP64 DDA: the primary answer. */
static void trace_one(const grid_t* G, const float* rf, or_hit* out) {
    ray64 R;
    memset(out, 0, sizeof(*out));
    out->x = out->y = out->z = -1;
    out->t = INFINITY;
    if (!load_ray(rf, &R)) { out->status = ST_INVALID; return; }
    double te, tx;
    int e;
    if (!root_slab(G, &R, &te, &tx, &e) || !(te < tx)) { out->status = ST_MISS; return; }
    int64_t v[3];
    start_voxel(G, &R, te, e, v);
    int64_t step[3];
    for (int i = 0; i < 3; i++) step[i] = R.d[i] > 0.0 ? 1 : (R.d[i] < 0.0 ? -1 : 0);
    double tcur = te;
    int face = e >= 0 ? face_of(&R, e) : 0;
    for (;;) {
        uint32_t w = gval(G, v);
        if (w != 0) {
            out->status = ST_HIT;
            out->t = tcur;
            out->rgba = w;
            out->x = (int32_t)v[0]; out->y = (int32_t)v[1]; out->z = (int32_t)v[2];
            out->face = face;
            return;
        }
        double tn[3];
        for (int i = 0; i < 3; i++) tn[i] = t_cross(&R, i, v[i]);
        int a = 0;
        if (tn[1] < tn[a]) a = 1;
        if (tn[2] < tn[a]) a = 2;
        tcur = tn[a];
        if (!(tcur < tx)) { out->status = ST_MISS; return; }
        v[a] += step[a];
        if (v[a] < 0 || v[a] >= G->n[a]) { out->status = ST_MISS; return; }
        face = face_of(&R, a);
    }
}

/* ------------------------------------------------------------------------ */
/* Near-tie classifier                                                       */
/*                                                                           */
/* Two crossings (or a crossing and the exit) whose times differ by less     */
/* than eps = eps_rel * max(n) / |d| -- the volume extent scaled by eps_rel  */
/* and converted to t -- may be taken in either order by an implementation   */
/* that rounds differently.  Walk every such order (a depth-first search     */
/* over voxels, each voxel expanded once, since a voxel's future depends     */
/* only on the voxel) and collect every reachable outcome.  A ray is a tie   */
/* when more than one outcome is reachable; non-consequential near-ties      */
/* (whose alternative voxels are all empty) do not make a tie.               */
/* ------------------------------------------------------------------------ */
#define OR_MAX_ALT 16

typedef struct {
    int32_t tie;      /* 1 when more than one outcome is reachable */
    int32_t n_alt;    /* distinct outcomes recorded (<= OR_MAX_ALT) */
    int32_t overflow; /* 1: outcome list full; 2: explored-state cap hit */
    int32_t pad;
    int64_t alt[OR_MAX_ALT];   /* voxel linear index, or -1 = MISS */
    double alt_t[OR_MAX_ALT];  /* entry t of that outcome (inf for MISS) */
} or_tie;

typedef struct {
    int64_t v[3];
    double t;
} wstate;

typedef struct {
    int64_t* keys;
    uint32_t* stamp;
    uint32_t cap_mask;
    uint32_t cur;
    wstate* stack;
    int64_t stack_cap;
    int64_t max_states;
} wspace;

static void ws_init(wspace* W, int log2cap, int64_t max_states) {
    uint32_t cap = 1u << log2cap;
    W->keys = (int64_t*)malloc(sizeof(int64_t) * cap);
    W->stamp = (uint32_t*)calloc(cap, sizeof(uint32_t));
    W->cap_mask = cap - 1;
    W->cur = 0;
    W->stack_cap = 4 * max_states + 64;
    W->stack = (wstate*)malloc(sizeof(wstate) * W->stack_cap);
    W->max_states = max_states;
}

static void ws_free(wspace* W) {
    free(W->keys); free(W->stamp); free(W->stack);
}

/* Returns 1 if key was newly inserted. */
static int ws_insert(wspace* W, int64_t key) {
    uint64_t h = (uint64_t)key * 0x9E3779B97F4A7C15ull;
    uint32_t i = (uint32_t)(h >> 40) & W->cap_mask;
    for (;;) {
        if (W->stamp[i] != W->cur) { W->stamp[i] = W->cur; W->keys[i] = key; return 1; }
        if (W->keys[i] == key) return 0;
        i = (i + 1) & W->cap_mask;
    }
}

static void add_outcome(or_tie* T, int64_t key, double t) {
    for (int i = 0; i < T->n_alt; i++)
        if (T->alt[i] == key) { if (t < T->alt_t[i]) T->alt_t[i] = t; return; }
    if (T->n_alt == OR_MAX_ALT) { T->overflow |= 1; return; }
    T->alt[T->n_alt] = key;
    T->alt_t[T->n_alt] = t;
    T->n_alt++;
}

static void classify_one(const grid_t* G, const float* rf, double eps_rel, or_tie* T, wspace* W) {
    memset(T, 0, sizeof(*T));
    ray64 R;
    if (!load_ray(rf, &R)) { add_outcome(T, -1, INFINITY); return; }
    double dn = sqrt(R.d[0] * R.d[0] + R.d[1] * R.d[1] + R.d[2] * R.d[2]);
    int64_t nmax = G->n[0];
    if (G->n[1] > nmax) nmax = G->n[1];
    if (G->n[2] > nmax) nmax = G->n[2];
    double eps = dn > 0.0 ? eps_rel * (double)nmax / dn : 0.0;
    double te, tx;
    int e;
    if (!root_slab(G, &R, &te, &tx, &e)) { add_outcome(T, -1, INFINITY); return; }
    if (!(te < tx)) {
        add_outcome(T, -1, INFINITY);
        if (!(te < tx + eps)) return;
    } else if (!(tx - te >= eps)) {
        add_outcome(T, -1, INFINITY);
    }
    int64_t step[3];
    for (int i = 0; i < 3; i++) step[i] = R.d[i] > 0.0 ? 1 : (R.d[i] < 0.0 ? -1 : 0);

    /* Start voxels: the primary one, plus the cell on the other side of any
     * voxel plane that the entry point lies within eps (in t) of. */
    int64_t v0[3];
    start_voxel(G, &R, te, e, v0);
    int64_t choice[3][2];
    int nch[3];
    for (int i = 0; i < 3; i++) {
        choice[i][0] = v0[i];
        nch[i] = 1;
        if (i == e || R.d[i] == 0.0) continue;
        double p = R.o[i] + te * R.d[i];
        double k = floor(p + 0.5);
        double tk = (k - R.o[i]) / R.d[i];
        if (fabs(tk - te) < eps) {
            int64_t ki = (int64_t)k, alt = -1;
            if (v0[i] == ki) alt = ki - 1;
            else if (v0[i] == ki - 1) alt = ki;
            if (alt >= 0 && alt < G->n[i]) { choice[i][1] = alt; nch[i] = 2; }
        }
    }
    W->cur++;
    if (W->cur == 0) { memset(W->stamp, 0, sizeof(uint32_t) * (W->cap_mask + 1)); W->cur = 1; }
    int64_t sp = 0, explored = 0;
    for (int a = 0; a < nch[0]; a++)
        for (int b = 0; b < nch[1]; b++)
            for (int c = 0; c < nch[2]; c++) {
                wstate s = {{choice[0][a], choice[1][b], choice[2][c]}, te};
                W->stack[sp++] = s;
            }
    while (sp > 0) {
        wstate s = W->stack[--sp];
        if (!ws_insert(W, glin(G, s.v))) continue;
        if (++explored > W->max_states) { T->overflow |= 2; break; }
        if (gval(G, s.v) != 0) { add_outcome(T, glin(G, s.v), s.t); continue; }
        double tn[3];
        for (int i = 0; i < 3; i++) tn[i] = t_cross(&R, i, s.v[i]);
        double m = tx;
        for (int i = 0; i < 3; i++) if (tn[i] < m) m = tn[i];
        if (isinf(m)) { add_outcome(T, -1, INFINITY); continue; }
        for (int i = 0; i < 3; i++) {
            if (R.d[i] == 0.0 || !(tn[i] - m < eps)) continue;
            wstate n = s;
            n.v[i] += step[i];
            n.t = tn[i];
            if (n.v[i] < 0 || n.v[i] >= G->n[i]) { add_outcome(T, -1, INFINITY); continue; }
            if (sp >= W->stack_cap) { T->overflow |= 2; continue; }
            W->stack[sp++] = n;
        }
        if (tx - m < eps) add_outcome(T, -1, INFINITY);
    }
    T->tie = T->n_alt > 1;
}

/* ------------------------------------------------------------------------ */
/* Brute force: slab-test the ray against every occupied voxel box.          */
/* "proper": the closed box is crossed over a t-interval of length >= eps;   */
/* "near": touched or missed by less than eps (interval length in            */
/* (-eps, eps), or a zero-direction axis on a box face).                     */
/* Acceptable outcomes: proper boxes entered within eps of the earliest      */
/* proper entry, near boxes entered no later than that plus eps, and MISS    */
/* when no box is proper.  Degenerate: more than one acceptable outcome.     */
/* ------------------------------------------------------------------------ */
typedef struct {
    int32_t hit;
    int32_t x, y, z;
    double t;
    int32_t degenerate;
    int32_t n_acc;    /* acceptable outcomes recorded */
    int64_t acc[16];  /* voxel linear index, or -1 = MISS */
} or_bf;

static void brute_one(const grid_t* G, const float* rf, double eps_rel, or_bf* B) {
    memset(B, 0, sizeof(*B));
    B->x = B->y = B->z = -1;
    B->t = INFINITY;
    ray64 R;
    if (!load_ray(rf, &R)) { B->n_acc = 1; B->acc[0] = -1; return; }
    double dn = sqrt(R.d[0] * R.d[0] + R.d[1] * R.d[1] + R.d[2] * R.d[2]);
    int64_t nmax = G->n[0];
    if (G->n[1] > nmax) nmax = G->n[1];
    if (G->n[2] > nmax) nmax = G->n[2];
    double eps = dn > 0.0 ? eps_rel * (double)nmax / dn : 0.0;
    double best = INFINITY;
    int64_t bestv[3] = {-1, -1, -1};
    int64_t v[3];
    /* pass 1: earliest proper entry */
    for (int pass = 0; pass < 2; pass++) {
        for (v[2] = 0; v[2] < G->n[2]; v[2]++)
            for (v[1] = 0; v[1] < G->n[1]; v[1]++)
                for (v[0] = 0; v[0] < G->n[0]; v[0]++) {
                    if (gval(G, v) == 0) continue;
                    double tn = R.tmin, tf = R.tmax;
                    int outside = 0, graze = 0;
                    for (int i = 0; i < 3; i++) {
                        double lo = (double)v[i], hi = (double)(v[i] + 1);
                        if (R.d[i] == 0.0) {
                            if (R.o[i] < lo || R.o[i] > hi) outside = 1;
                            else if (R.o[i] == lo || R.o[i] == hi) graze = 1;
                            continue;
                        }
                        double a = ((R.d[i] > 0.0 ? lo : hi) - R.o[i]) / R.d[i];
                        double b = ((R.d[i] > 0.0 ? hi : lo) - R.o[i]) / R.d[i];
                        if (a > tn) tn = a;
                        if (b < tf) tf = b;
                    }
                    if (outside) continue;
                    int proper = !graze && (tf - tn >= eps);
                    int nearb = !proper && (tf - tn > -eps);
                    if (pass == 0) {
                        if (proper && tn < best) {
                            best = tn;
                            bestv[0] = v[0]; bestv[1] = v[1]; bestv[2] = v[2];
                        }
                    } else {
                        int acc = (proper && tn <= best + eps) || (nearb && tn <= best + eps);
                        if (acc && B->n_acc < 16) B->acc[B->n_acc++] = glin(G, v);
                    }
                }
    }
    if (bestv[0] >= 0) {
        B->hit = 1;
        B->x = (int32_t)bestv[0]; B->y = (int32_t)bestv[1]; B->z = (int32_t)bestv[2];
        B->t = best;
    } else if (B->n_acc < 16) {
        B->acc[B->n_acc++] = -1;
    }
    B->degenerate = B->n_acc > 1;
}

/* ------------------------------------------------------------------------ */
/* Pinhole camera, FP64, rounded once to float32 at the end.                 */
/* cam = {eye[3], look[3], up[3], vfov_deg}.  Pixel (px, py), py = 0 at the  */
/* top row, samples its centre: sx = (2 (px + 0.5) / W - 1) tan(fov/2) W/H,  */
/* sy = (1 - 2 (py + 0.5) / H) tan(fov/2); d = normalize(f + sx r + sy u)    */
/* with f = normalize(look - eye), r = normalize(f x up), u = r x f.         */
/* Ray i = px + W py: {eye, 0, d, +inf}.                                     */
/* ------------------------------------------------------------------------ */
static void norm3(double v[3]) {
    double l = sqrt(v[0] * v[0] + v[1] * v[1] + v[2] * v[2]);
    v[0] /= l; v[1] /= l; v[2] /= l;
}

void or_pinhole(const double* cam, int64_t W, int64_t H, float* rays) {
    const double PI = 3.14159265358979323846264338327950288;
    double f[3] = {cam[3] - cam[0], cam[4] - cam[1], cam[5] - cam[2]};
    norm3(f);
    const double* up = cam + 6;
    double r[3] = {f[1] * up[2] - f[2] * up[1], f[2] * up[0] - f[0] * up[2], f[0] * up[1] - f[1] * up[0]};
    norm3(r);
    double u[3] = {r[1] * f[2] - r[2] * f[1], r[2] * f[0] - r[0] * f[2], r[0] * f[1] - r[1] * f[0]};
    double th = tan(cam[9] * PI / 360.0);
    double aspect = (double)W / (double)H;
    for (int64_t py = 0; py < H; py++)
        for (int64_t px = 0; px < W; px++) {
            double sx = (2.0 * ((double)px + 0.5) / (double)W - 1.0) * th * aspect;
            double sy = (1.0 - 2.0 * ((double)py + 0.5) / (double)H) * th;
            double d[3];
            for (int i = 0; i < 3; i++) d[i] = f[i] + sx * r[i] + sy * u[i];
            norm3(d);
            float* o = rays + 8 * (px + W * py);
            o[0] = (float)cam[0]; o[1] = (float)cam[1]; o[2] = (float)cam[2];
            o[3] = 0.0f;
            o[4] = (float)d[0]; o[5] = (float)d[1]; o[6] = (float)d[2];
            o[7] = INFINITY;
        }
}

/* ------------------------------------------------------------------------ */
/* Decoder of the paper's word-buffer layout (Sec. 3.3, Fig. 3) into a       */
/* dense grid.  Format signatures follow Table 1 with log2 extents:          */
/* R(W,H,D) a 2^W x 2^H x 2^D array of terminating integers; S(L) an octree  */
/* of depth L; G(L) a DAG of depth L; "N^3" is shorthand for N,N,N.          */
/* Word 0 is the pointer to the root sub-volume (0 = empty volume).          */
/*   Raw:  2^(W+H+D) words, cell (x,y,z) at x + (y << W) + (z << (W+H)).     */
/*   SVO node: {first-child pointer or terminating integer, masks}; masks =  */
/*         valid | leaf << 8; valid children stored contiguously, 2 words    */
/*         each, in child-index order (child i = x | y << 1 | z << 2).       */
/*   SVDAG node: {masks or terminating integer, one pointer per valid        */
/*         child}; a leaf node is one terminating-integer word.              */
/*   DF D(W,H,D,M): a Raw grid with a second word per cell, interleaved     */
/*         {terminating integer, l1}: cell (x,y,z) at 2 (x + (y << W) +      */
/*         (z << (W+H))).  l1 is the L1 (Manhattan) distance, in cells, from  */
/*         the cell to the nearest non-empty cell of the same sub-volume,    */
/*         capped at M (0 for a non-empty cell) (Sec. 3.1, 3.3, 4.1).        */
/* A terminating integer is a word offset of a next-level sub-volume, or the */
/* voxel RGBA at the last level; 0 = empty.                                  */
/* Returns 0, or a negative code: -1 bad spec, -2 pointer out of range,      */
/* -3 inconsistent masks, -4 voxel outside the grid, -5 empty valid child,   */
/* -6 unsupported level kind, -7 a DF distance differs from its definition.  */
/* ------------------------------------------------------------------------ */
typedef struct {
    char kind;
    int e[3];
    int param;
} dlevel;

static int parse_spec(const char* s, dlevel* lv, int maxlv) {
    int n = 0;
    while (*s) {
        while (*s == ' ' || *s == '\t' || *s == ',') s++;
        if (!*s) break;
        char k = *s++;
        if (k != 'R' && k != 'S' && k != 'G' && k != 'D') return -1;
        while (*s == ' ') s++;
        if (*s++ != '(') return -1;
        int vals[4], nv = 0;
        for (;;) {
            while (*s == ' ') s++;
            if (*s < '0' || *s > '9') return -1;
            int x = 0;
            while (*s >= '0' && *s <= '9') x = 10 * x + (*s++ - '0');
            while (*s == ' ') s++;
            if (*s == '^') {
                s++;
                if (*s++ != '3' || nv + 3 > 4) return -1;
                vals[nv++] = x; vals[nv++] = x; vals[nv++] = x;
            } else {
                if (nv >= 4) return -1;
                vals[nv++] = x;
            }
            while (*s == ' ') s++;
            if (*s == ',') { s++; continue; }
            if (*s == ')') { s++; break; }
            return -1;
        }
        if (n >= maxlv) return -1;
        dlevel* L = &lv[n++];
        L->kind = k;
        L->param = 0;
        if (k == 'R') {
            if (nv != 3) return -1;
            L->e[0] = vals[0]; L->e[1] = vals[1]; L->e[2] = vals[2];
        } else if (k == 'D') {
            if (nv != 4) return -1;
            L->e[0] = vals[0]; L->e[1] = vals[1]; L->e[2] = vals[2]; L->param = vals[3];
        } else {
            if (nv != 1 || vals[0] < 1) return -1;
            L->e[0] = L->e[1] = L->e[2] = vals[0];
        }
    }
    return n;
}

typedef struct {
    const uint32_t* w;
    uint64_t nw;
    uint32_t* grid;
    int64_t n[3];
    dlevel lv[32];
    int nlv;
    int s[32][3]; /* log2 cell size of level k per axis */
    int err;
} dctx;

static void dec_level(dctx* C, int k, uint32_t ptr, int64_t lo[3]);

static void dec_emit(dctx* C, int k, uint32_t term, int64_t lo[3]) {
    if (k == C->nlv - 1) {
        for (int i = 0; i < 3; i++)
            if (lo[i] < 0 || lo[i] >= C->n[i]) { C->err = -4; return; }
        C->grid[lo[0] + C->n[0] * (lo[1] + C->n[1] * lo[2])] = term;
    } else {
        dec_level(C, k + 1, term, lo);
    }
}

static void dec_svo(dctx* C, int k, uint32_t np, int depth, int64_t lo[3]) {
    if (C->err) return;
    const dlevel* L = &C->lv[k];
    if ((uint64_t)np + 2 > C->nw || np == 0) { C->err = -2; return; }
    uint32_t first = C->w[np], masks = C->w[np + 1];
    uint32_t valid = masks & 0xFFu, leaf = (masks >> 8) & 0xFFu;
    int last = depth == L->e[0] - 1;
    if ((masks >> 16) != 0 || valid == 0 || leaf != (last ? valid : 0u)) { C->err = -3; return; }
    int64_t half = (int64_t)1 << (C->s[k][0] + L->e[0] - depth - 1);
    uint32_t rank = 0;
    for (int i = 0; i < 8 && !C->err; i++) {
        if (!((valid >> i) & 1u)) continue;
        uint64_t c = (uint64_t)first + 2ull * rank++;
        int64_t cl[3] = {lo[0] + (i & 1) * half, lo[1] + ((i >> 1) & 1) * half, lo[2] + ((i >> 2) & 1) * half};
        if (last) {
            if (c + 2 > C->nw) { C->err = -2; return; }
            uint32_t term = C->w[c];
            if (term == 0) { C->err = -5; return; }
            if (C->w[c + 1] != 0) { C->err = -3; return; }
            dec_emit(C, k, term, cl);
        } else {
            if (c > 0xFFFFFFFFull) { C->err = -2; return; }
            dec_svo(C, k, (uint32_t)c, depth + 1, cl);
        }
    }
}

static void dec_dag(dctx* C, int k, uint32_t np, int depth, int64_t lo[3]) {
    if (C->err) return;
    const dlevel* L = &C->lv[k];
    if ((uint64_t)np + 1 > C->nw || np == 0) { C->err = -2; return; }
    uint32_t masks = C->w[np];
    uint32_t valid = masks & 0xFFu, leaf = (masks >> 8) & 0xFFu;
    int last = depth == L->e[0] - 1;
    if ((masks >> 16) != 0 || valid == 0 || leaf != (last ? valid : 0u)) { C->err = -3; return; }
    int64_t half = (int64_t)1 << (C->s[k][0] + L->e[0] - depth - 1);
    uint32_t rank = 0;
    for (int i = 0; i < 8 && !C->err; i++) {
        if (!((valid >> i) & 1u)) continue;
        uint64_t slot = (uint64_t)np + 1 + rank++;
        if (slot >= C->nw) { C->err = -2; return; }
        uint32_t cp = C->w[slot];
        int64_t cl[3] = {lo[0] + (i & 1) * half, lo[1] + ((i >> 1) & 1) * half, lo[2] + ((i >> 2) & 1) * half};
        if (last) {
            if (cp == 0 || (uint64_t)cp >= C->nw) { C->err = -2; return; }
            uint32_t term = C->w[cp];
            if (term == 0) { C->err = -5; return; }
            dec_emit(C, k, term, cl);
        } else {
            dec_dag(C, k, cp, depth + 1, cl);
        }
    }
}

/* The distance of DF cell c: the smallest L1 distance to a non-empty cell of
 * the sub-volume, capped at M.  Written out directly: the minimum over the
 * list of non-empty cells, or over the cells within L1 distance M of c,
 * whichever list is shorter (both give the definition). */
static uint32_t df_distance(const uint32_t* cells, const int e[3], int64_t M, const int64_t* occ, int64_t nocc,
                            int64_t cx, int64_t cy, int64_t cz) {
    const int64_t nx = (int64_t)1 << e[0], ny = (int64_t)1 << e[1], nz = (int64_t)1 << e[2];
    int64_t best = M;
    const int64_t ball = (2 * M + 1) * (2 * M + 1) * (2 * M + 1);
    if (nocc <= ball) {
        for (int64_t q = 0; q < nocc; q++) {
            const int64_t x = occ[q] % nx, y = (occ[q] / nx) % ny, z = occ[q] / (nx * ny);
            const int64_t d = llabs(x - cx) + llabs(y - cy) + llabs(z - cz);
            if (d < best) best = d;
        }
    } else {
        for (int64_t dz = -M; dz <= M; dz++)
            for (int64_t dy = -M; dy <= M; dy++)
                for (int64_t dx = -M; dx <= M; dx++) {
                    const int64_t d = llabs(dx) + llabs(dy) + llabs(dz);
                    if (d >= best) continue;
                    const int64_t x = cx + dx, y = cy + dy, z = cz + dz;
                    if (x < 0 || y < 0 || z < 0 || x >= nx || y >= ny || z >= nz) continue;
                    if (cells[2 * (x + nx * (y + ny * z))] != 0) best = d;
                }
    }
    return (uint32_t)best;
}

static void dec_df(dctx* C, int k, uint32_t ptr, int64_t lo[3]) {
    const dlevel* L = &C->lv[k];
    const int64_t nx = (int64_t)1 << L->e[0], ny = (int64_t)1 << L->e[1], nz = (int64_t)1 << L->e[2];
    const int64_t cnt = nx * ny * nz;
    if ((uint64_t)ptr + 2ull * (uint64_t)cnt > C->nw) { C->err = -2; return; }
    const uint32_t* cells = C->w + ptr;  /* cell i: cells[2 i] terminating integer, cells[2 i + 1] distance */
    int64_t nocc = 0;
    for (int64_t i = 0; i < cnt; i++) nocc += cells[2 * i] != 0;
    int64_t* occ = (int64_t*)malloc(sizeof(int64_t) * (size_t)(nocc > 0 ? nocc : 1));
    nocc = 0;
    for (int64_t i = 0; i < cnt; i++)
        if (cells[2 * i] != 0) occ[nocc++] = i;
    for (int64_t z = 0; z < nz && !C->err; z++)
        for (int64_t y = 0; y < ny && !C->err; y++)
            for (int64_t x = 0; x < nx && !C->err; x++) {
                const int64_t i = x + nx * (y + ny * z);
                const uint32_t w = cells[2 * i];
                const uint32_t want = w != 0 ? 0u : df_distance(cells, L->e, L->param, occ, nocc, x, y, z);
                if (cells[2 * i + 1] != want) { C->err = -7; break; }
                if (w == 0) continue;
                int64_t cl[3] = {lo[0] + (x << C->s[k][0]), lo[1] + (y << C->s[k][1]), lo[2] + (z << C->s[k][2])};
                dec_emit(C, k, w, cl);
            }
    free(occ);
}

static void dec_level(dctx* C, int k, uint32_t ptr, int64_t lo[3]) {
    if (C->err) return;
    const dlevel* L = &C->lv[k];
    if (ptr == 0) { C->err = -2; return; }
    if (L->kind == 'R') {
        uint64_t cnt = 1ull << (L->e[0] + L->e[1] + L->e[2]);
        if ((uint64_t)ptr + cnt > C->nw) { C->err = -2; return; }
        for (int64_t z = 0; z < (1 << L->e[2]); z++)
            for (int64_t y = 0; y < (1 << L->e[1]); y++)
                for (int64_t x = 0; x < (1 << L->e[0]); x++) {
                    uint32_t w = C->w[ptr + x + (y << L->e[0]) + (z << (L->e[0] + L->e[1]))];
                    if (w == 0) continue;
                    int64_t cl[3] = {lo[0] + (x << C->s[k][0]), lo[1] + (y << C->s[k][1]), lo[2] + (z << C->s[k][2])};
                    dec_emit(C, k, w, cl);
                    if (C->err) return;
                }
    } else if (L->kind == 'S') {
        dec_svo(C, k, ptr, 0, lo);
    } else if (L->kind == 'G') {
        dec_dag(C, k, ptr, 0, lo);
    } else if (L->kind == 'D') {
        dec_df(C, k, ptr, lo);
    } else {
        C->err = -6;
    }
}

/* Fills grid (caller zeroes it, dims must equal the spec's total extents). */
int or_decode(const uint32_t* words, uint64_t nwords, const char* spec, uint32_t* grid,
              int64_t nx, int64_t ny, int64_t nz) {
    dctx* C = (dctx*)calloc(1, sizeof(dctx));
    C->w = words; C->nw = nwords; C->grid = grid;
    C->n[0] = nx; C->n[1] = ny; C->n[2] = nz;
    C->nlv = parse_spec(spec, C->lv, 32);
    if (C->nlv <= 0) { free(C); return -1; }
    int tot[3] = {0, 0, 0};
    for (int k = C->nlv - 1; k >= 0; k--)
        for (int i = 0; i < 3; i++) { C->s[k][i] = tot[i]; tot[i] += C->lv[k].e[i]; }
    for (int i = 0; i < 3; i++)
        if (((int64_t)1 << tot[i]) != C->n[i]) { free(C); return -1; }
    int rc = 0;
    if (nwords < 1) rc = -2;
    else if (words[0] != 0) {
        int64_t lo[3] = {0, 0, 0};
        dec_level(C, 0, words[0], lo);
        rc = C->err;
    }
    free(C);
    return rc;
}

/* Dimensions (log2 per axis) implied by a spec; returns number of levels or -1. */
int or_spec_dims(const char* spec, int32_t* log2dims) {
    dlevel lv[32];
    int n = parse_spec(spec, lv, 32);
    if (n <= 0) return -1;
    log2dims[0] = log2dims[1] = log2dims[2] = 0;
    for (int k = 0; k < n; k++)
        for (int i = 0; i < 3; i++) log2dims[i] += lv[k].e[i];
    return n;
}

/* ------------------------------------------------------------------------ */
/* Threaded drivers                                                          */
/* ------------------------------------------------------------------------ */
typedef struct {
    const grid_t* G;
    const float* rays;
    int64_t begin, end;
    int mode; /* 0 trace, 1 classify, 2 brute */
    double eps_rel;
    void* out;
} job_t;

static void* run_job(void* p) {
    job_t* J = (job_t*)p;
    if (J->mode == 0) {
        or_hit* out = (or_hit*)J->out;
        for (int64_t r = J->begin; r < J->end; r++) trace_one(J->G, J->rays + 8 * r, out + r);
    } else if (J->mode == 1) {
        or_tie* out = (or_tie*)J->out;
        wspace W;
        ws_init(&W, 17, 1 << 15);
        for (int64_t r = J->begin; r < J->end; r++) classify_one(J->G, J->rays + 8 * r, J->eps_rel, out + r, &W);
        ws_free(&W);
    } else {
        or_bf* out = (or_bf*)J->out;
        for (int64_t r = J->begin; r < J->end; r++) brute_one(J->G, J->rays + 8 * r, J->eps_rel, out + r);
    }
    return NULL;
}

static int run_threads(const grid_t* G, const float* rays, int64_t n, int mode, double eps_rel, void* out,
                       int nthreads) {
    if (nthreads < 1) nthreads = 1;
    if (nthreads > 256) nthreads = 256;
    if (n < 4096 * nthreads) {
        int64_t t = n / 4096;
        nthreads = t < 1 ? 1 : (int)(t < nthreads ? t : nthreads);
    }
    pthread_t th[256];
    job_t jobs[256];
    /* Interleaved chunks balance cost across threads. */
    for (int i = 0; i < nthreads; i++) {
        jobs[i].G = G; jobs[i].rays = rays; jobs[i].mode = mode; jobs[i].eps_rel = eps_rel; jobs[i].out = out;
        jobs[i].begin = n * i / nthreads;
        jobs[i].end = n * (i + 1) / nthreads;
    }
    for (int i = 1; i < nthreads; i++) pthread_create(&th[i], NULL, run_job, &jobs[i]);
    run_job(&jobs[0]);
    for (int i = 1; i < nthreads; i++) pthread_join(th[i], NULL);
    return nthreads;
}

static void make_grid(grid_t* G, const uint32_t* g32, const uint8_t* g8, const uint32_t* pal, int64_t nx,
                      int64_t ny, int64_t nz) {
    G->g32 = g32; G->g8 = g8; G->pal = pal;
    G->n[0] = nx; G->n[1] = ny; G->n[2] = nz;
}

/* Public entry points.  grid: nx*ny*nz RGBA words (x fastest).  rays: n x 8
 * floats.  Each returns the number of threads it used. */
int or_trace(const uint32_t* grid, int64_t nx, int64_t ny, int64_t nz, const float* rays, int64_t n, or_hit* out,
             int nthreads) {
    grid_t G;
    make_grid(&G, grid, NULL, NULL, nx, ny, nz);
    return run_threads(&G, rays, n, 0, 0.0, out, nthreads);
}

/* Same, for a grid of 8-bit palette indices (palette[0] must be 0). */
int or_trace_pal(const uint8_t* grid, const uint32_t* palette, int64_t nx, int64_t ny, int64_t nz,
                 const float* rays, int64_t n, or_hit* out, int nthreads) {
    grid_t G;
    make_grid(&G, NULL, grid, palette, nx, ny, nz);
    return run_threads(&G, rays, n, 0, 0.0, out, nthreads);
}

int or_classify(const uint32_t* grid, int64_t nx, int64_t ny, int64_t nz, const float* rays, int64_t n,
                double eps_rel, or_tie* out, int nthreads) {
    grid_t G;
    make_grid(&G, grid, NULL, NULL, nx, ny, nz);
    return run_threads(&G, rays, n, 1, eps_rel, out, nthreads);
}

int or_classify_pal(const uint8_t* grid, const uint32_t* palette, int64_t nx, int64_t ny, int64_t nz,
                    const float* rays, int64_t n, double eps_rel, or_tie* out, int nthreads) {
    grid_t G;
    make_grid(&G, NULL, grid, palette, nx, ny, nz);
    return run_threads(&G, rays, n, 1, eps_rel, out, nthreads);
}

int or_bruteforce(const uint32_t* grid, int64_t nx, int64_t ny, int64_t nz, const float* rays, int64_t n,
                  double eps_rel, or_bf* out, int nthreads) {
    grid_t G;
    make_grid(&G, grid, NULL, NULL, nx, ny, nz);
    return run_threads(&G, rays, n, 2, eps_rel, out, nthreads);
}

int or_sizeof(int which) {
    switch (which) {
        case 0: return (int)sizeof(or_hit);
        case 1: return (int)sizeof(or_tie);
        case 2: return (int)sizeof(or_bf);
        default: return -1;
    }
}

/* ------------------------------------------------------------------------ */
/* Ambient-occlusion rays (FP64, rounded once to float32).                   */
/* For primary ray i with a hit on face f (1 + 2a + s, a = axis, s = 1 when  */
/* the ray moved towards -a): the outward normal of the entered face is     */
/* n = -e_a (s = 0) or +e_a (s = 1); sample k of spp draws two uniforms      */
/* u1, u2 from SplitMix64 (Steele, Lea & Flood 2014) of the counter          */
/* c = (i * spp + k) * 2 + {0, 1} mixed with the seed, keeping the top 24    */
/* bits; Malley's method: a uniform point on the unit disk, r = sqrt(u1),    */
/* phi = 2 pi u2, lifted to the hemisphere, z = sqrt(1 - u1): a cosine-      */
/* weighted direction d = r cos(phi) e_{a+1} + r sin(phi) e_{a+2} + z n      */
/* (axes mod 3).  Origin: the hit point o + t d_primary moved eps along n;   */
/* tmin 0, tmax = tmax_ao.  Misses and face-0 hits give the empty ray        */
/* {0,0,0, 0, 0,0,0, 0}.  Output ray i * spp + k.                            */
/* ------------------------------------------------------------------------ */
static uint64_t ao_mix(uint64_t x) {
    x += 0x9E3779B97F4A7C15ull;
    x = (x ^ (x >> 30)) * 0xBF58476D1CE4E5B9ull;
    x = (x ^ (x >> 27)) * 0x94D049BB133111EBull;
    return x ^ (x >> 31);
}

static double ao_u24(uint64_t seed, uint64_t c) {
    uint64_t h = ao_mix(ao_mix(seed) ^ c);
    return (double)(h >> 40) / 16777216.0;
}

void or_ao_rays(const float* rays, const or_hit* hits, int64_t n, uint64_t seed, int spp, double eps, double tmax_ao,
                float* out) {
    const double PI = 3.14159265358979323846264338327950288;
    for (int64_t i = 0; i < n; i++) {
        const or_hit* h = &hits[i];
        for (int k = 0; k < spp; k++) {
            float* o = out + 8 * (i * spp + k);
            if (h->status != ST_HIT || h->face == 0) {
                for (int q = 0; q < 8; q++) o[q] = 0.0f;
                continue;
            }
            const int a = (h->face - 1) / 2, s = (h->face - 1) & 1;
            const double sign = s ? 1.0 : -1.0;
            const uint64_t c = ((uint64_t)i * (uint64_t)spp + (uint64_t)k) * 2u;
            const double u1 = ao_u24(seed, c), u2 = ao_u24(seed, c + 1);
            const double r = sqrt(u1), phi = 2.0 * PI * u2;
            const double lx = r * cos(phi), ly = r * sin(phi), lz = sqrt(1.0 - u1 > 0.0 ? 1.0 - u1 : 0.0);
            double d[3] = {0, 0, 0}, p[3];
            d[(a + 1) % 3] = lx;
            d[(a + 2) % 3] = ly;
            d[a] = sign * lz;
            const float* pr = rays + 8 * i;
            for (int q = 0; q < 3; q++) p[q] = (double)pr[q] + h->t * (double)pr[4 + q];
            p[a] += sign * eps;
            o[0] = (float)p[0]; o[1] = (float)p[1]; o[2] = (float)p[2];
            o[3] = 0.0f;
            o[4] = (float)d[0]; o[5] = (float)d[1]; o[6] = (float)d[2];
            o[7] = (float)tmax_ao;
        }
    }
}
