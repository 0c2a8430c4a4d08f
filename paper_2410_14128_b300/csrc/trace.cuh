// trace.cuh -- first-hit traversal of a hybrid voxel format on sm_103a.
//
// What it computes (Sec. 4.2): the root function reads the root pointer from
// word 0, tests the ray against the root box and enters level 1; each level
// visits the non-empty children its ray crosses in hit-time order and hands
// the first non-empty one to the next level (Fig. 4, intersect /
// ordered_hit_children); the answer is the first occupied voxel.
//
// How (a B300 design, not the paper's GLSL):
//   * All levels share one loop.  The format is expanded into node levels
//     (fmt.hpp); the ray keeps the integer coordinate of the cell it is in
//     at the current node level, and a short stack of node pointers, one per
//     level.  Each iteration either looks the current cell up (and descends
//     into it when it is non-empty) or takes one Amanatides-Woo step to the
//     neighbouring cell of the same level (Sec. 2; Raw levels are a plain
//     grid DDA, octree nodes are a 2x2x2 grid), so lanes of a warp execute
//     the same instructions whatever level each is at.  Stepping out of a
//     node resumes at the deepest ancestor that still contains the new cell
//     (the highest changed coordinate bit selects it), so no level ever
//     re-walks its parent.
//   * Raw lookups read cell x + (y << W) + (z << (W+H)); octree children are
//     found from the valid mask with popc: the child list of an SVO node is
//     contiguous (first + 2 rank), an SVDAG node lists one pointer per valid
//     child (node[1 + rank]) (Sec. 3.3, Fig. 3).
//   * Every boundary crossing is computed in closed form from the integer
//     plane, t = (plane - o) / d, in FP32.  Whenever two FP32 quantities that
//     decide a step lie within 2^-20 (relative) of each other -- 16x the
//     worst FP32 error of those expressions -- the decision is re-taken in
//     FP64 with exactly the expressions of the FP64 reference stepper
//     (lowest axis first on equality).  So the voxel found equals that of a
//     plain FP64 DDA over the uncompressed grid, not just within a tolerance.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include "fmt.hpp"

namespace vx {

constexpr float kGuard = 9.5367431640625e-07f;  // 2^-20

// Resident blocks of 256 threads per SM the kernels are compiled for
// (64 registers a thread, some spills).  Measured on the 512^3 terrain step:
// persistent kernels at 4 beat 3 (80 registers) by 1.7%, and 3 beats 2;
// the one-ray-per-thread kernels at 4 beat the unconstrained build (80
// registers) by 7-11% on primary rays.
#ifndef VX_PERSIST_MINB
#define VX_PERSIST_MINB 4
#endif
#ifndef VX_PLAIN_MINB
#define VX_PLAIN_MINB 4
#endif
#define VX_PLAIN_BOUNDS __launch_bounds__(256, VX_PLAIN_MINB)

enum : uint32_t { ST_MISS = 0, ST_HIT = 1, ST_INVALID = 2, ST_ERROR = 3 };

// ---------------------------------------------------------------------------
// Format accessors: run-time (kernel argument) and compile-time (template).
// ---------------------------------------------------------------------------
struct DynF {
    FmtParams p;
    static constexpr int kMaxJ = kMaxNodeLevels;
    __device__ __forceinline__ int J() const { return (int)p.J; }
    __device__ __forceinline__ int kind(int j) const { return (int)((p.kind >> (2 * j)) & 3u); }
    __device__ __forceinline__ int s(int j) const { return (int)((p.s >> (4 * j)) & 15u); }
    __device__ __forceinline__ int b(int j) const { return (int)((p.b >> (4 * j)) & 15u); }
    __device__ __forceinline__ bool bot(int j) const { return (p.bot >> j) & 1u; }
    __device__ __forceinline__ uint32_t top() const { return p.top; }
    __device__ __forceinline__ int b0(int a) const { return (int)p.b0[a]; }
    __device__ __forceinline__ int ldim(int a) const { return (int)p.ldim[a]; }
    __device__ __forceinline__ int jpop(int h) const { return (int)((p.jpop >> (4 * h)) & 15u); }
    __device__ __forceinline__ bool has_svo() const { return true; }
    __device__ __forceinline__ bool has_dag() const { return true; }
    __device__ __forceinline__ bool has_df() const { return true; }
};

template <uint32_t J_, uint32_t KIND, uint32_t BOT, uint64_t S, uint64_t B, uint32_t B0X, uint32_t B0Y, uint32_t B0Z,
          uint32_t LX, uint32_t LY, uint32_t LZ, uint64_t JPOP, uint32_t TOP>
struct StatF {
    static constexpr int kMaxJ = (int)J_;
    __device__ __forceinline__ int J() const { return (int)J_; }
    __device__ __forceinline__ int kind(int j) const { return (int)((KIND >> (2 * j)) & 3u); }
    // 4-bit fields of the packed 64-bit constants; a 32-bit shift when the
    // fields a walk can index fit the low word (J <= 8 node levels, grids of
    // at most 2^8 per axis for jpop), a 64-bit funnel shift otherwise
    __device__ __forceinline__ int s(int j) const {
        return J_ <= 8 ? (int)(((uint32_t)S >> (4 * j)) & 15u) : (int)((S >> (4 * j)) & 15u);
    }
    __device__ __forceinline__ int b(int j) const {
        return J_ <= 8 ? (int)(((uint32_t)B >> (4 * j)) & 15u) : (int)((B >> (4 * j)) & 15u);
    }
    __device__ __forceinline__ bool bot(int j) const { return (BOT >> j) & 1u; }
    __device__ __forceinline__ uint32_t top() const { return TOP; }
    __device__ __forceinline__ int b0(int a) const { return (int)(a == 0 ? B0X : (a == 1 ? B0Y : B0Z)); }
    __device__ __forceinline__ int ldim(int a) const { return (int)(a == 0 ? LX : (a == 1 ? LY : LZ)); }
    __device__ __forceinline__ int jpop(int h) const {
        constexpr uint32_t kMaxL = LX > LY ? (LX > LZ ? LX : LZ) : (LY > LZ ? LY : LZ);
        return kMaxL <= 8 ? (int)(((uint32_t)JPOP >> (4 * h)) & 15u) : (int)((JPOP >> (4 * h)) & 15u);
    }
    static constexpr bool kHasSvo = (KIND & 0x55555555u & ~(KIND >> 1)) != 0;
    static constexpr bool kHasDag = ((KIND >> 1) & 0x55555555u & ~KIND) != 0;
    static constexpr bool kHasDf = (KIND & (KIND >> 1) & 0x55555555u) != 0;
    __device__ __forceinline__ bool has_svo() const { return kHasSvo; }
    __device__ __forceinline__ bool has_dag() const { return kHasDag; }
    __device__ __forceinline__ bool has_df() const { return kHasDf; }
};

// Compile-time composition: Format<Raw<4,4,4>, Svo<2>, Dag<3>>.
template <int W, int H, int D>
struct Raw {
    static constexpr LevelDesc desc() { return LevelDesc{K_RAW, {W, H, D}}; }
};
// D(W,H,D,M): the cap M is a property of the stored distances, not of the
// traversal, so the kernel does not depend on it.
template <int W, int H, int D, int M>
struct Df {
    static constexpr LevelDesc desc() { return LevelDesc{K_DF, {W, H, D}}; }
};
template <int L>
struct Svo {
    static constexpr LevelDesc desc() { return LevelDesc{K_SVO, {L, L, L}}; }
};
template <int L>
struct Dag {
    static constexpr LevelDesc desc() { return LevelDesc{K_DAG, {L, L, L}}; }
};

template <class... Ls>
struct Format {
    static constexpr FmtParams make() {
        FmtParams p{};
        LevelDesc lv[] = {Ls::desc()...};
        make_fmt_params(lv, (int)sizeof...(Ls), &p);
        return p;
    }
    static constexpr FmtParams P = make();
    static_assert(P.J > 0, "format cannot be composed");
    using F = StatF<P.J, P.kind, P.bot, P.s, P.b, P.b0[0], P.b0[1], P.b0[2], P.ldim[0], P.ldim[1], P.ldim[2], P.jpop,
                    P.top>;
};

// ---------------------------------------------------------------------------
// Ray input and hit record
// ---------------------------------------------------------------------------
struct RayIn {
    float o[3];
    float tmin;
    float d[3];
    float tmax;
};

struct HitRec {
    float t;
    uint32_t rgba;
    int x, y, z;
    int face;
    uint32_t status;
};

// Per-ray work counters of the instrumented kernels: words of the format
// read (in bytes), loop iterations, and decisions re-taken in FP64.
struct Cnt {
    uint32_t bytes = 0, iters = 0, fp64 = 0;
    uint32_t refused = 0;  // reads outside the image, refused (instrumented kernels check every read)
};

__device__ __forceinline__ HitRec miss_rec(uint32_t st) {
    HitRec h;
    h.t = __int_as_float(0x7f800000);
    h.rgba = 0;
    h.x = h.y = h.z = 0xFFFF;
    h.face = 0;
    h.status = st;
    return h;
}

// ---------------------------------------------------------------------------
// FP64 decisions (rare; kept out of line).  Each expression is the one the
// FP64 reference stepper evaluates, one IEEE rounding per operation.
// ---------------------------------------------------------------------------
__device__ __forceinline__ double t64(float o, float d, int plane) {
    return __ddiv_rn(__dsub_rn((double)plane, (double)o), (double)d);
}

struct Root64 {
    double te, tx;
    int e;
};

// Root slab test in FP64.  Axes with d == 0 were checked by the caller.
// (Scalar arguments: a struct argument would force the ray into local memory.)
static __device__ __noinline__ Root64 root64(float o0, float o1, float o2, float d0, float d1, float d2, float tmin,
                                             float tmax, int l0, int l1, int l2) {
    const float o[3] = {o0, o1, o2}, d[3] = {d0, d1, d2};
    const int ld[3] = {l0, l1, l2};
    double best = -__longlong_as_double(0x7ff0000000000000ll);
    double tx = (double)tmax;
    int e = -1;
#pragma unroll
    for (int i = 0; i < 3; i++) {
        if (d[i] == 0.0f) continue;
        const int n = 1 << ld[i];
        const int lo = d[i] > 0.0f ? 0 : n;
        const int hi = d[i] > 0.0f ? n : 0;
        const double a = t64(o[i], d[i], lo);
        const double b = t64(o[i], d[i], hi);
        if (a > best) { best = a; e = i; }
        if (b < tx) tx = b;
    }
    Root64 R;
    if (e >= 0 && best > (double)tmin) { R.te = best; R.e = e; }
    else { R.te = (double)tmin; R.e = -1; }
    R.tx = tx;
    return R;
}

// Start voxel coordinate on a non-entry axis from the FP64 entry point.
static __device__ __noinline__ int start_coord64(float o, float d, double te) {
    const double p = __dadd_rn((double)o, __dmul_rn(te, (double)d));
    double f = floor(p);
    f = fmin(fmax(f, -2.0), 65536.0);
    int v = (int)f;
    if (p == f && d < 0.0f) v -= 1;
    return v;
}

// Which of the crossing candidates comes first in FP64 (lowest axis on ties).
static __device__ __noinline__ int argmin64(float o0, float o1, float o2, float d0, float d1, float d2, int p0, int p1,
                                            int p2) {
    const float o[3] = {o0, o1, o2}, d[3] = {d0, d1, d2};
    const int pl[3] = {p0, p1, p2};
    int a = -1;
    double m = 0.0;
#pragma unroll
    for (int i = 0; i < 3; i++) {
        if (d[i] == 0.0f) continue;
        const double t = t64(o[i], d[i], pl[i]);
        if (a < 0 || t < m) { m = t; a = i; }
    }
    return a;
}

// Is the crossing time tc (FP64) at or after the exit?
// (The exit does not depend on tmin, so the walk need not keep it.)
static __device__ __noinline__ bool exits64(float o0, float o1, float o2, float d0, float d1, float d2, float tmax,
                                            int l0, int l1, int l2, float oa, float da, int plane) {
    const Root64 R = root64(o0, o1, o2, d0, d1, d2, 0.0f, tmax, l0, l1, l2);
    return !(t64(oa, da, plane) < R.tx);
}

// Has the ray crossed plane B on axis a before the crossing of plane lp on
// axis la that brought it into the current cell?
static __device__ __noinline__ bool crossed64(float oa, float da, int B, int a, float ol, float dl, int lp, int la) {
    const double tb = t64(oa, da, B);
    const double tc = t64(ol, dl, lp);
    return tb < tc || (tb == tc && a < la);
}

// Element i of a 3-array, by selects: a runtime index into a small array
// would move the array to local memory.
template <class T>
__device__ __forceinline__ T sel3(const T (&v)[3], int i) {
    return i == 0 ? v[0] : (i == 1 ? v[1] : v[2]);
}

__device__ __forceinline__ bool near32(float x, float y) {
    return !(fabsf(x - y) > kGuard * fmaxf(fabsf(x), fabsf(y)));
}

__device__ __forceinline__ uint32_t ldw(const uint32_t* __restrict__ pool, uint32_t i) { return __ldg(pool + i); }

// A volume's device image: its words, whether they are in the packed layout
// (pack.cpp: pointers to SVDAG nodes carry the node's valid mask in bits
// 24..31; SVDAG slots of leaf children hold the terminating integer), and
// whether two-word structures start at even words (then {pointer, masks} of
// an SVO node and {terminating integer, distance} of a DF cell are one
// 8-byte load).
struct Img {
    const uint32_t* w;
    int packed;
    uint32_t n;   // words in the image (the instrumented kernels check every read against it)
    int aligned;  // DF cell arrays, SVO root entries and SVO child lists start at even words
};
constexpr uint32_t kPtrMask = 0x00FFFFFFu;

// ---------------------------------------------------------------------------
// The traversal
// ---------------------------------------------------------------------------
#define VX_CNT(field, v)            \
    do {                            \
        if (COUNT) cnt.field += (v); \
    } while (0)

// The traversal state of one ray.  start() does the root part (validity,
// slab test, start voxel, root node); step() runs one iteration of the loop
// (one cell lookup with its descent, or one Amanatides-Woo step with its
// pop).  Both return true once the ray is finished, with the record in `out`.
// Keeping the state between calls lets a warp swap finished rays for new ones
// without leaving the loop (persistent kernels).
//
// The node stack (pointer and valid mask of the node entered at each node
// level, one 8-byte entry per level, and the start voxel) lives in the
// kernel's dynamic shared memory (vx_dyn_smem below), one column per thread.
//
// SMODE selects how nodes are resumed after a step leaves a node:
//   0  full stack: one entry per node level, every node entered is kept;
//   1  the paper's restarting sparse-voxel intersection (Sec. 4.4): only the
//      root node of each format level is kept; leaving a node of an SVO or
//      SVDAG level walks that level's octree again from its root down to the
//      resuming node level, at the price of re-reading those nodes;
//   2  short stack: the format levels' roots, plus the nodes of the other
//      (octree) node levels in a ring of D = sdm + 1 entries indexed by
//      j mod D and tagged with their level; a pop whose entry was overwritten
//      by a deeper level falls back to the restart of mode 1.
//
// TOPS: the calling kernel copied the first `stw` words of the device image
// into shared memory (after the node stacks); the relocated image holds the
// structures of its top node levels there, level by level (pack.cpp), so
// every read below word stw -- the top k node levels of any kind -- comes
// from shared memory.
//
// Dynamic shared memory of every walker kernel: first the node stacks of the
// block's threads, entry e of thread t at vx_dyn_smem[t * stack_stride(J) +
// e] (8-byte entries), then, in a persistent kernel that stages the top
// level, its words.  The stride is odd, so the 16 lanes of a half-warp that
// read the same entry touch 16 distinct 8-byte bank pairs (no bank
// conflicts), and a thread reaches any entry from one base register plus a
// constant; the stack takes no L1 lines from node reads.
extern __shared__ __align__(16) uint2 vx_dyn_smem[];
constexpr uint32_t kTopSmemMaxWords = 8192;  // 32 KiB of staged image words at most

// Shared-memory carveout preference of a walker kernel, in percent of the
// SM's maximum (228 KiB): what its resident blocks need (the kernels are
// compiled for 1024 resident threads per SM), so that the rest of the SM's
// on-chip memory stays L1 for node reads.  Set once per kernel and value
// (launch.cu).
void prefer_carveout(const void* kernel, size_t smem_per_block, int block);

// Entries per thread: one {pointer, valid mask} per node level, then two
// holding values a walk reads rarely -- {start voxel x, y}, {start voxel z,
// tmax} -- which would otherwise take registers; the stride rounds that up to
// an odd count.  A short stack (mode 2) adds its ring of D entries after
// those.
__host__ __device__ constexpr uint32_t stack_entries(uint32_t J, uint32_t D = 0) { return J + 2u + D; }
__host__ __device__ constexpr uint32_t stack_stride(uint32_t J, uint32_t D = 0) { return stack_entries(J, D) | 1u; }
inline size_t stack_bytes(uint32_t J, int block, uint32_t D = 0) {
    return (size_t)stack_stride(J, D) * (size_t)block * sizeof(uint2);
}
constexpr int kShortStackMax = 8;  // ring depths 1, 2, 4, 8

template <bool COUNT, class F, int SMODE = 0, bool TOPS = false>
struct Walker {
    RayIn r;
    float inv[3];
    float tx, tcur;
    float gabs;  // guard band: 2^-20 of the largest |t| this walk compares
    // (direction sign per axis, -1 / 0 / 1: sgn(), from the ray)
    int c[3];  // cell at node level j (the start voxel is kept in the stack array)
    float gpos;  // guard band for positions o + t d inside the grid (read by descents)
    int j, la, budget;
    int skip;  // DF level: cells the walk may still enter without a look-up
    bool fresh;
    uint32_t Pc, Mc;  // node of level j: pointer, valid mask
    uint32_t sb;      // shared-window byte address of this thread's stack entry 0
    uint32_t sdm = 0;  // short stack (SMODE 2): ring depth - 1, a power of two minus one
    uint32_t stw = 0;  // TOPS: words of the image staged in shared memory
    uint32_t lim;     // words in the image (checked by the instrumented walker)
    uint32_t* sect;   // instrumented walker: one bit per 32-byte sector of the image it read, or null
    Cnt cnt;

    // A word of the image.  The instrumented walker (COUNT) checks every
    // index against the image size and refuses reads outside it (counted; the
    // ray then reports ST_ERROR), so it can walk a buffer nobody validated;
    // it also marks the 32-byte sector (8 words) each accepted read falls in.
    __device__ __forceinline__ uint32_t rd(const uint32_t* __restrict__ pool, uint32_t i) {
        if (TOPS && i < stw) return staged_words()[i];
        if (COUNT) {
            if (i >= lim) {
                cnt.refused++;
                return 0u;
            }
            if (sect) atomicOr(sect + (i >> 8), 1u << ((i >> 3) & 31u));
        }
        return ldw(pool, i);
    }

    // Words i and i + 1 of the image (an SVO node entry, a DF cell): one
    // 8-byte load when the image is aligned (i is then even), else two.
    __device__ __forceinline__ uint2 rd2(const Img& im, uint32_t i) {
        if (TOPS && i + 1u < stw) return make_uint2(staged_words()[i], staged_words()[i + 1u]);
        if (COUNT) {
            if (i + 1u >= lim || i + 1u < i || (im.aligned && (i & 1u))) {
                cnt.refused++;
                return make_uint2(0u, 0u);
            }
            if (sect) atomicOr(sect + (i >> 8), 1u << ((i >> 3) & 31u));
        }
        if (im.aligned) return __ldg(reinterpret_cast<const uint2*>(im.w + i));
        return make_uint2(ldw(im.w, i), ldw(im.w, i + 1u));
    }


    // Node-stack entry e of this thread (0 <= e < stack_entries(J); entries
    // J and J + 1 hold the start voxel and tmax).  Every index the walk forms lies in
    // that range by construction (j only grows by descents below J - 1 and
    // pops to jpop(h) <= j); the instrumented walker also checks it and
    // refuses an access outside it (counted like a refused read).
    __device__ __forceinline__ uint32_t saddr(const F& f, int e) {
        if (COUNT && (unsigned)e >= stack_entries((uint32_t)f.J(), ring())) {
            cnt.refused++;
            e = 0;
        }
        return sb + 8u * (uint32_t)e;
    }
    __device__ __forceinline__ uint32_t ring() const { return SMODE == 2 ? sdm + 1u : 0u; }
    __device__ __forceinline__ uint2 sget(const F& f, int e) {
        uint2 v;
        asm volatile("ld.shared.v2.u32 {%0, %1}, [%2];" : "=r"(v.x), "=r"(v.y) : "r"(saddr(f, e)));
        return v;
    }
    __device__ __forceinline__ void sput(const F& f, int e, uint2 v) {
        asm volatile("st.shared.v2.u32 [%0], {%1, %2};" ::"r"(saddr(f, e)), "r"(v.x), "r"(v.y) : "memory");
    }
    // the staged image words (TOPS kernels run with SMODE 0: no ring)
    __device__ __forceinline__ const uint32_t* staged_words() const { return reinterpret_cast<const uint32_t*>(vx_dyn_smem) + 2u * sbase_words; }
    uint32_t sbase_words = 0;  // TOPS: 8-byte entries before the staged words (stacks of the block)

    // Node level j: kind, children side (log2 voxels), fanout per axis, and
    // whether its children are terminating integers -- extracted from the
    // format's constants each time (measured: cheaper than keeping copies in
    // registers, which spill).
    __device__ __forceinline__ int lk(const F& f) const { return f.kind(j); }
    __device__ __forceinline__ int ls(const F& f) const { return f.s(j); }
    __device__ __forceinline__ int lb(const F& f, int a) const { return j == 0 ? f.b0(a) : f.b(j); }
    __device__ __forceinline__ bool lbot(const F& f) const { return f.bot(j); }

    __device__ __forceinline__ int sgn(int i) const {
        const float d = sel3(r.d, i);
        return d > 0.0f ? 1 : (d < 0.0f ? -1 : 0);
    }

    // Node of level j reached from the root of its format level: the nodes
    // on the way are ancestors of the cell the walk just left, so each exists.
    // Node level d's child holding cell c (side 2^s_j) has index bit
    // (c >> (s_d - s_j)) & 1 per axis.
    __device__ __forceinline__ void restart(const F& f, const Img im) {
        const uint32_t* __restrict__ pool = im.w;
        const int r = 31 - __clz(f.top() & ((2u << j) - 1u));
        const uint2 e = sget(f, r);
        uint32_t p = e.x, m = e.y;
        const bool svo = f.has_svo() && f.kind(r) == K_SVO;
        const int sj = f.s(j);
        for (int d = r; d < j; d++) {
            const int sh = f.s(d) - sj;
            const uint32_t idx = ((uint32_t)(c[0] >> sh) & 1u) | (((uint32_t)(c[1] >> sh) & 1u) << 1) |
                                 (((uint32_t)(c[2] >> sh) & 1u) << 2);
            const uint32_t rank = __popc(m & ((1u << idx) - 1u));
            if (svo) {
                const uint2 e2 = rd2(im, p + 2u * rank);
                p = e2.x;
                m = e2.y & 0xFFu;
                VX_CNT(bytes, 8);
            } else {
                const uint32_t cp = rd(pool, p + 1u + rank);
                if (im.packed) { p = cp & kPtrMask; m = cp >> 24; VX_CNT(bytes, 4); }
                else { p = cp; m = rd(pool, cp) & 0xFFu; VX_CNT(bytes, 8); }
            }
        }
        Pc = p;
        Mc = m;
    }

    // |x - y| within the guard band (true for NaN: decide in FP64)
    __device__ __forceinline__ bool near(float x, float y) const { return !(fabsf(x - y) > gabs); }

    __device__ __forceinline__ bool start(const F& f, const Img im, const RayIn& ray, HitRec& out) {
        const uint32_t* __restrict__ pool = im.w;
        lim = im.n;
        sb = (uint32_t)__cvta_generic_to_shared(vx_dyn_smem) + 8u * stack_stride((uint32_t)f.J(), ring()) * threadIdx.x;
        r = ray;
        // Invalid rays: any NaN, or an infinite tmin.
        if (isnan(r.o[0]) || isnan(r.o[1]) || isnan(r.o[2]) || isnan(r.d[0]) || isnan(r.d[1]) || isnan(r.d[2]) ||
            isnan(r.tmin) || isnan(r.tmax) || isinf(r.tmin)) {
            out = miss_rec(ST_INVALID);
            return true;
        }
        float nf[3];
#pragma unroll
        for (int i = 0; i < 3; i++) {
            inv[i] = __frcp_rn(r.d[i]);
            nf[i] = (float)(1 << f.ldim(i));
        }

        // ---- root slab test (FP32, FP64 when undecided) ----
        float t0[3], best = -__int_as_float(0x7f800000);
        tx = r.tmax;
        int e = -1;
#pragma unroll
        for (int i = 0; i < 3; i++) {
            t0[i] = 0.0f;
            if (sgn(i) == 0) {
                if (!(r.o[i] >= 0.0f && r.o[i] < nf[i])) {
                    out = miss_rec(ST_MISS);
                    return true;
                }
                continue;
            }
            const float lo = sgn(i) > 0 ? 0.0f : nf[i];
            const float hi = sgn(i) > 0 ? nf[i] : 0.0f;
            t0[i] = (lo - r.o[i]) * inv[i];
            const float t1 = (hi - r.o[i]) * inv[i];
            if (t0[i] > best) { best = t0[i]; e = i; }
            tx = fminf(tx, t1);
        }
        bool unsure = false;
#pragma unroll
        for (int i = 0; i < 3; i++)
            if (sgn(i) != 0 && i != e && near32(t0[i], best)) unsure = true;
        if (e >= 0 && near32(best, r.tmin)) unsure = true;
        int ea;
        float te;
        if (e >= 0 && best > r.tmin) { te = best; ea = e; }
        else { te = r.tmin; ea = -1; }
        bool miss;
        if (unsure || near32(te, tx)) {
            VX_CNT(fp64, 1);
            const Root64 R = root64(r.o[0], r.o[1], r.o[2], r.d[0], r.d[1], r.d[2], r.tmin, r.tmax, f.ldim(0),
                                    f.ldim(1), f.ldim(2));
            ea = R.e;
            te = (float)R.te;
            tx = (float)R.tx;
            miss = !(R.te < R.tx);
        } else {
            miss = !(te < tx);
        }
        if (miss) {
            out = miss_rec(ST_MISS);
            return true;
        }

        // ---- start voxel ----
        int v0l[3];
#pragma unroll
        for (int i = 0; i < 3; i++) {
            const int n = 1 << f.ldim(i);
            int v;
            if (i == ea) {
                v = sgn(i) > 0 ? 0 : n - 1;
            } else {
                const float p = fmaf(te, r.d[i], r.o[i]);
                const float fl = floorf(p);
                v = (int)fminf(fmaxf(fl, -2.0f), 65536.0f);
                if (sgn(i) != 0) {
                    const float rq = rintf(p);
                    if (fabsf(p - rq) <= kGuard * (fabsf(te * r.d[i]) + fabsf(p))) {
                        VX_CNT(fp64, 1);
                        const double te64 = ea >= 0 ? t64(sel3(r.o, ea), sel3(r.d, ea),
                                                          sgn(ea) > 0 ? 0 : (1 << f.ldim(ea)))
                                                    : (double)r.tmin;
                        v = start_coord64(r.o[i], r.d[i], te64);
                    }
                }
            }
            v0l[i] = min(max(v, 0), n - 1);
        }
        // the start voxel is read only by descents before the first step and
        // by the FP64 tie rule: it lives in the stack's two extra entries,
        // not in registers
        sput(f, f.J(), make_uint2((uint32_t)v0l[0], (uint32_t)v0l[1]));
        sput(f, f.J() + 1, make_uint2((uint32_t)v0l[2], __float_as_uint(r.tmax)));

        // ---- root node ----
        const uint32_t root = rd(pool, 0);
        VX_CNT(bytes, 4);
        if (root == 0) {
            out = miss_rec(ST_MISS);
            return true;
        }
        {
            const int k0 = f.kind(0);
            if (k0 == K_RAW || k0 == K_DF) { Pc = root; Mc = 0; }
            else if (k0 == K_SVO) { const uint2 e2 = rd2(im, root); Pc = e2.x; Mc = e2.y & 0xFFu; VX_CNT(bytes, 8); }
            else if (im.packed) { Pc = root & kPtrMask; Mc = root >> 24; }
            else { Pc = root; Mc = rd(pool, root) & 0xFFu; VX_CNT(bytes, 4); }
        }
        j = 0;
        sput(f, 0, make_uint2(Pc, Mc));
        {
            const int s0 = f.s(0);
#pragma unroll
            for (int i = 0; i < 3; i++) c[i] = v0l[i] >> s0;
        }
        la = ea;  // axis of the last crossing
        tcur = te;
        fresh = true;  // no step taken yet
        // Every crossing this walk compares lies in [min(te, tx), max(te, tx)]
        // (crossings past the exit end it), and the FP32 error of one is at
        // most 3 2^-24 |t|: a band of 2^-20 max|t| covers both operands 16x.
        gabs = kGuard * fmaxf(fabsf(te), fabsf(tx));
        // o + t d (FP32) is off by at most |d| 3 2^-24 |t| + 2^-24 |p|, with
        // |t| <= max(|te|, |tx|) and |p| within the grid where it matters.
        gpos = gabs * fmaxf(fabsf(r.d[0]), fmaxf(fabsf(r.d[1]), fabsf(r.d[2]))) +
               kGuard * (float)(2 << max(f.ldim(0), max(f.ldim(1), f.ldim(2))));
        // A ray crosses at most nx + ny + nz cells of any level and each step
        // costs at most J descents; past this bound the ray reports ST_ERROR.
        budget = ((1 << f.ldim(0)) + (1 << f.ldim(1)) + (1 << f.ldim(2)) + 4) * (f.J() + 2);
        skip = 0;
        return false;
    }

    // One Amanatides-Woo step at node level j, with the pop when the step
    // leaves the node.  Returns true once the ray is finished (out holds the
    // miss).
    __device__ __forceinline__ bool advance(const F& f, const Img im, HitRec& out) {
        if (r.d[0] == 0.0f && r.d[1] == 0.0f && r.d[2] == 0.0f) {
            out = miss_rec(ST_MISS);
            return true;
        }
        // next plane per axis and its crossing, in closed form from the cell
        int pl[3];
        float tn[3];
#pragma unroll
        for (int i = 0; i < 3; i++) {
            pl[i] = (c[i] + (sgn(i) > 0 ? 1 : 0)) << ls(f);
            tn[i] = sgn(i) != 0 ? ((float)pl[i] - r.o[i]) * inv[i] : __int_as_float(0x7f800000);
        }
        int a = tn[1] < tn[0] ? 1 : 0;
        float tm = fminf(tn[0], tn[1]);
        if (tn[2] < tm) { a = 2; tm = tn[2]; }
        // second smallest crossing; a d = 0 axis (+inf) is never near
        const float t2 = fminf(fmaxf(tn[0], tn[1]), fmaxf(fminf(tn[0], tn[1]), tn[2]));
        const bool und = !(t2 - tm > gabs);
        if (und) {
            VX_CNT(fp64, 1);
            a = argmin64(r.o[0], r.o[1], r.o[2], r.d[0], r.d[1], r.d[2], pl[0], pl[1], pl[2]);
            tm = sel3(tn, a);
        }
        // A step through the grid's boundary ends the walk whatever the exit
        // comparison says; only an exit on another axis or at tmax can tie.
        const int pla = sel3(pl, a), sga = sgn(a);
        bool out_now = pla == (sga > 0 ? (1 << f.ldim(a)) : 0);
        if (!out_now) {
            if (near(tm, tx)) {
                VX_CNT(fp64, 1);
                const float tmax = __uint_as_float(sget(f, f.J() + 1).y);
                out_now = exits64(r.o[0], r.o[1], r.o[2], r.d[0], r.d[1], r.d[2], tmax, f.ldim(0), f.ldim(1),
                                  f.ldim(2), sel3(r.o, a), sel3(r.d, a), pla);
            } else {
                out_now = !(tm < tx);
            }
        }
        if (out_now) {
            out = miss_rec(ST_MISS);
            return true;
        }
        const int old = sel3(c, a);
        const int nw = old + sga;
#pragma unroll
        for (int i = 0; i < 3; i++)
            if (i == a) c[i] = nw;
        tcur = tm;
        la = a;
        fresh = false;
        const int h = 31 - __clz((uint32_t)(old ^ nw)) + ls(f);  // highest changed voxel-coordinate bit
        const int span = j == 0 ? f.ldim(a) : f.s(j - 1);
        if (h >= span) {
            skip = 0;  // the distances are those of the node the walk left
            if (h >= f.ldim(a)) {
                out = miss_rec(ST_MISS);
                return true;
            }
            const int jp = f.jpop(h);
            const int sh = f.s(jp) - ls(f);
#pragma unroll
            for (int i = 0; i < 3; i++) c[i] >>= sh;
            j = jp;
            if (SMODE == 1) {
                restart(f, im);
            } else if (SMODE == 2 && !((f.top() >> j) & 1u)) {
                const uint2 e = sget(f, f.J() + 2 + (j & (int)sdm));
                if ((e.y >> 8) == (uint32_t)(j + 1)) {
                    Pc = e.x;
                    Mc = e.y & 0xFFu;
                } else {
                    restart(f, im);  // overwritten by a deeper level of the ring
                }
            } else {
                const uint2 e = sget(f, j);
                Pc = e.x;
                Mc = e.y;
            }
        }
        return false;
    }

    __device__ __forceinline__ bool step(const F& f, const Img im, HitRec& out) {
        const uint32_t* __restrict__ pool = im.w;
        if (--budget < 0) {
            out = miss_rec(ST_ERROR);
            return true;
        }
        VX_CNT(iters, 1);
        const int J = f.J();
        const int kind = lk(f);
        const int bx = lb(f, 0), by = lb(f, 1), bz = lb(f, 2);
        const uint32_t lx = (uint32_t)c[0] & ((1u << bx) - 1u);
        const uint32_t ly = (uint32_t)c[1] & ((1u << by) - 1u);
        const uint32_t lz = (uint32_t)c[2] & ((1u << bz) - 1u);
        // child index: x + (y << W) + (z << (W+H)) for Raw; the same formula
        // gives x | y << 1 | z << 2 inside an octree node (W = H = D = 1)
        const uint32_t idx = lx | (ly << bx) | (lz << (bx + by));
        // The look-up is written without divergent branches (loads under a
        // predicate, results by selects): lanes at different kinds of level,
        // or DF lanes that skip and lanes that read, stay together and reach
        // the step below as one group.
        const bool is_raw = kind == K_RAW;
        const bool is_df = f.has_df() && kind == K_DF;
        // DF cell {terminating integer, L1 distance d}: every cell within L1
        // distance d - 1 is empty, and each Amanatides-Woo step moves one cell
        // along one axis, so the next d - 1 cells of the walk at this level
        // are entered without reading them (Sec. 4.2).
        const bool df_read = is_df && skip <= 0;
        const uint32_t a = is_df ? Pc + 2u * idx : Pc + idx;
        uint32_t w = 0, dist = 0;
        if (!COUNT && !TOPS && f.has_df() && im.aligned) {
            // one 8-byte load for lanes at DF and at Raw levels alike: a DF
            // cell {terminating integer, distance} starts at an even word; a
            // Raw cell is the half of its aligned pair that the parity picks
            // (the image ends on an even word, so the pair is inside it)
            if (is_raw || df_read) {
                const uint2 v = __ldg(reinterpret_cast<const uint2*>(pool + (a & ~1u)));
                w = (a & 1u) ? v.y : v.x;
                dist = v.y;
            }
        } else {
            if (is_raw || df_read) w = rd(pool, a);
            if (df_read) dist = rd(pool, a + 1);  // same sector as the cell word
        }
        VX_CNT(bytes, is_raw ? 4 : (df_read ? 8 : 0));
        const bool occ = (is_raw || is_df) ? w != 0u : ((Mc >> idx) & 1u) != 0u;
        if (is_df) skip = df_read ? (occ ? 0 : (int)dist - 1) : skip - 1;
        if (occ) {
            // ---- descend (or hit at the last node level) ----
            uint32_t term = w, Pn = 0, Mn = 0;
            bool node_ready = false;
            if (kind == K_SVO || kind == K_DAG) {
                const uint32_t rank = __popc(Mc & ((1u << idx) - 1u));
                if (f.has_svo() && kind == K_SVO) {
                    const uint32_t addr = Pc + 2u * rank;
                    if (lbot(f)) { term = rd(pool, addr); VX_CNT(bytes, 4); }
                    else { const uint2 e2 = rd2(im, addr); Pn = e2.x; Mn = e2.y & 0xFFu; node_ready = true; VX_CNT(bytes, 8); }
                } else {
                    const uint32_t cp = rd(pool, Pc + 1u + rank);
                    if (im.packed) {
                        if (lbot(f)) term = cp;
                        else { Pn = cp & kPtrMask; Mn = cp >> 24; node_ready = true; }
                        VX_CNT(bytes, 4);
                    } else {
                        if (lbot(f)) term = rd(pool, cp);
                        else { Pn = cp; Mn = rd(pool, cp) & 0xFFu; node_ready = true; }
                        VX_CNT(bytes, 8);
                    }
                }
            }
            if (j == J - 1) {
                out.t = tcur;
                out.rgba = term;
                out.x = c[0]; out.y = c[1]; out.z = c[2];
                out.face = la >= 0 ? 1 + 2 * la + (sgn(la) < 0 ? 1 : 0) : 0;
                out.status = ST_HIT;
                return true;
            }
            if (!node_ready) {
                const int nk = f.kind(j + 1);
                if (nk == K_RAW || nk == K_DF) { Pn = term; }
                else if (f.has_svo() && nk == K_SVO) { const uint2 e2 = rd2(im, term); Pn = e2.x; Mn = e2.y & 0xFFu; VX_CNT(bytes, 8); }
                else if (im.packed) { Pn = term & kPtrMask; Mn = term >> 24; }
                else { Pn = term; Mn = rd(pool, term) & 0xFFu; VX_CNT(bytes, 4); }
            }
            ++j;
            if (SMODE == 0 || ((f.top() >> j) & 1u)) sput(f, j, make_uint2(Pn, Mn));
            else if (SMODE == 2) sput(f, J + 2 + (j & (int)sdm), make_uint2(Pn, Mn | ((uint32_t)(j + 1) << 8)));
            Pc = Pn;
            Mc = Mn;
            const int sn = ls(f), bn = lb(f, 0);
            const float scale = __int_as_float((127 - sn) << 23);  // 2^-sn
            if (fresh) {  // no step yet: the cell holding the start voxel
                const uint2 a01 = sget(f, J), a2 = sget(f, J + 1);
                c[0] = (int)a01.x >> sn;
                c[1] = (int)a01.y >> sn;
                c[2] = (int)a2.x >> sn;
                return false;
            }
#pragma unroll
            for (int i = 0; i < 3; i++) {
                const int base = c[i] << bn;
                const int topc = base + (1 << bn) - 1;
                if (i == la) { c[i] = sgn(i) > 0 ? base : topc; continue; }
                if (sgn(i) == 0) { c[i] = (int)floorf(r.o[i]) >> sn; continue; }  // o inside the grid on that axis
                const float p = fmaf(tcur, r.d[i], r.o[i]);
                const float q = p * scale;
                int cn = (int)fminf(fmaxf(floorf(q), (float)base), (float)topc);
                const float rq = rintf(q);
                if (rq > (float)base && rq <= (float)topc &&
                    fabsf(q - rq) <= gpos * scale) {
                    VX_CNT(fp64, 1);
                    const int B = (int)rq;
                    // plane of the crossing that entered the parent's cell (voxel units):
                    // the parent cell's face on axis la, from its coordinate (c[la]
                    // already holds the child's when la < i)
                    const int cpar = la < i ? (sel3(c, la) >> bn) : sel3(c, la);
                    const int lpl = (cpar + (sgn(la) < 0 ? 1 : 0)) << (sn + bn);
                    const bool cr = crossed64(r.o[i], r.d[i], B << sn, i, sel3(r.o, la), sel3(r.d, la), lpl, la);
                    cn = sgn(i) > 0 ? (cr ? B : B - 1) : (cr ? B - 1 : B);
                    // a ray that started on plane B took the start voxel's
                    // convention; a crossing at that same instant must not undo it
                    // (away from the band the cell is past the start anyway)
                    const uint2 sv = sget(f, i == 2 ? J + 1 : J);
                    const int vs = (int)(i == 1 ? sv.y : sv.x) >> sn;
                    cn = sgn(i) > 0 ? max(cn, vs) : min(cn, vs);
                }
                c[i] = cn;
            }
            return false;
        }

        // ---- one Amanatides-Woo step at node level j ----
        return advance(f, im, out);
    }
};
#undef VX_CNT

template <bool COUNT, class F, int SMODE = 0>
__device__ __forceinline__ HitRec trace_ray(const F& f, const Img pool, const RayIn& r, Cnt& cnt,
                                            uint32_t* sect = nullptr, uint32_t sdm = 0) {
    Walker<COUNT, F, SMODE> w;  // node stack in the kernel's dynamic shared memory
    w.sect = sect;
    w.sdm = sdm;
    HitRec h;
    if (!w.start(f, pool, r, h))
        while (!w.step(f, pool, h)) {
        }
    if (COUNT) {
        cnt.bytes += w.cnt.bytes;
        cnt.iters += w.cnt.iters;
        cnt.fp64 += w.cnt.fp64;
        cnt.refused += w.cnt.refused;
        if (w.cnt.refused) h = miss_rec(ST_ERROR);
    }
    return h;
}

// ---------------------------------------------------------------------------
// Hit stores
// ---------------------------------------------------------------------------
template <int LAYOUT, class F>
__device__ __forceinline__ void store_hit(const F& f, void* hits, uint64_t i, const HitRec& h) {
    if (LAYOUT == 0) {
        uint4 v;
        v.x = __float_as_uint(h.t);
        v.y = h.rgba;
        v.z = ((uint32_t)h.x & 0xFFFFu) | ((uint32_t)h.y << 16);
        v.w = ((uint32_t)h.z & 0xFFFFu) | ((uint32_t)h.face << 16) | (h.status << 24);
        __stcs(reinterpret_cast<uint4*>(hits) + i, v);
    } else {
        uint2 v;
        v.x = h.status == ST_HIT
                  ? (uint32_t)h.x + ((uint32_t)h.y << f.ldim(0)) + ((uint32_t)h.z << (f.ldim(0) + f.ldim(1)))
                  : 0xFFFFFFFFu;
        v.y = __float_as_uint(h.t);
        __stcs(reinterpret_cast<uint2*>(hits) + i, v);
    }
}

__device__ __forceinline__ RayIn load_ray(const float4* __restrict__ rays, uint64_t i) {
    const float4 a = __ldcs(rays + 2 * i);
    const float4 b = __ldcs(rays + 2 * i + 1);
    RayIn r;
    r.o[0] = a.x; r.o[1] = a.y; r.o[2] = a.z; r.tmin = a.w;
    r.d[0] = b.x; r.d[1] = b.y; r.d[2] = b.z; r.tmax = b.w;
    return r;
}

// ---------------------------------------------------------------------------
// Pinhole camera (FP32), pixel (px, py) through its centre.
// ---------------------------------------------------------------------------
struct CamDev {
    float eye[3], f[3], r[3], u[3];
    float tha, th;
    uint32_t W, H;
};

__device__ __forceinline__ RayIn pinhole_ray(const CamDev& c, uint32_t px, uint32_t py) {
    const float sx = (2.0f * ((float)px + 0.5f) / (float)c.W - 1.0f) * c.tha;
    const float sy = (1.0f - 2.0f * ((float)py + 0.5f) / (float)c.H) * c.th;
    float d[3];
#pragma unroll
    for (int i = 0; i < 3; i++) d[i] = c.f[i] + sx * c.r[i] + sy * c.u[i];
    const float inv = 1.0f / sqrtf(d[0] * d[0] + d[1] * d[1] + d[2] * d[2]);
    RayIn r;
#pragma unroll
    for (int i = 0; i < 3; i++) { r.o[i] = c.eye[i]; r.d[i] = d[i] * inv; }
    r.tmin = 0.0f;
    r.tmax = __int_as_float(0x7f800000);
    return r;
}

// ---------------------------------------------------------------------------
// Kernels
// ---------------------------------------------------------------------------
// Ray k of the launch writes hit k (a sorted trace runs on the sorted copies
// of the rays and hits, sort.cu).
template <class F, int LAYOUT, int SM = 0>
__global__ void VX_PLAIN_BOUNDS k_trace(F f, const Img pool, const float4* __restrict__ rays, uint64_t n,
                                               void* __restrict__ hits, uint32_t sdm) {
    const uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const RayIn r = load_ray(rays, i);
    Cnt cnt;
    const HitRec h = trace_ray<false, F, SM>(f, pool, r, cnt, nullptr, sdm);
    store_hit<LAYOUT>(f, hits, i, h);
}

// Instrumented twin of k_trace: same results, plus totals of the per-ray
// counters in counters[0..3] (bytes of the format read, iterations, FP64
// decisions, reads refused as outside the image), summed per warp then added
// atomically.  Every read of the image is checked against its size.
template <class F, int LAYOUT, bool RS = false>
__global__ void VX_PLAIN_BOUNDS k_trace_count(F f, const Img pool,
                                                     const float4* __restrict__ rays, uint64_t n,
                                                     void* __restrict__ hits, unsigned long long* counters,
                                                     uint32_t* sectors) {
    const uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
    Cnt cnt;
    if (i < n) {
        const RayIn r = load_ray(rays, i);
        const HitRec h = trace_ray<true, F, RS ? 1 : 0>(f, pool, r, cnt, sectors);
        store_hit<LAYOUT>(f, hits, i, h);
    }
    unsigned long long b = cnt.bytes, it = cnt.iters, d = cnt.fp64, rf = cnt.refused;
    for (int o = 16; o > 0; o >>= 1) {
        b += __shfl_down_sync(0xffffffffu, b, o);
        it += __shfl_down_sync(0xffffffffu, it, o);
        d += __shfl_down_sync(0xffffffffu, d, o);
        rf += __shfl_down_sync(0xffffffffu, rf, o);
    }
    if ((threadIdx.x & 31) == 0) {
        atomicAdd(counters + 0, b);
        atomicAdd(counters + 1, it);
        atomicAdd(counters + 2, d);
        atomicAdd(counters + 3, rf);
    }
}

constexpr uint32_t kTileW = 8, kTileH = 32 / kTileW;  // pixels of a warp's tile

// Persistent render: like k_trace_persistent, with the rays generated from
// the queue slots instead of read from memory.  Slot s is lane s % 32 of tile
// s / 32, the tiles of 8 x 4 pixels taken row by row over the image rows from
// y0 (the order of the plain render kernel's warps), so the lanes one refill
// hands out sit in one or two neighbouring tiles.  Slots of pixels outside
// the image or outside [i0, i0 + n) are taken and dropped.
template <class F, int LAYOUT>
__global__ void __launch_bounds__(256, VX_PERSIST_MINB) k_render_persistent(F f, const Img pool, CamDev cam, uint64_t i0,
                                                           uint64_t n, uint32_t y0, uint32_t tiles_w, uint64_t slots,
                                                           void* __restrict__ hits,
                                                           unsigned long long* next, int refill, int burst) {
    const unsigned lane = threadIdx.x & 31u;
    const unsigned lt_mask = (1u << lane) - 1u;
    Walker<false, F> w;  // node stack in the kernel's dynamic shared memory
    bool live = false;
    bool exhausted = false;  // warp-uniform
    uint64_t pix = 0;        // hit index (pixel - i0) of the lane's ray
    while (true) {
        const unsigned idle = __ballot_sync(0xffffffffu, !live);
        if (exhausted) {
            if (idle == 0xffffffffu) break;
        } else if (__popc(idle) >= refill) {
            const int leader = __ffs(idle) - 1;
            unsigned long long base = 0;
            if ((int)lane == leader) base = atomicAdd(next, (unsigned long long)__popc(idle));
            base = __shfl_sync(0xffffffffu, base, leader);
            if (base + (unsigned long long)__popc(idle) >= slots) exhausted = true;
            if (!live) {
                const uint64_t slot = base + __popc(idle & lt_mask);
                if (slot < slots) {
                    uint32_t trow, tcol;
                    if (slots < (1ull << 37)) {  // tile index below 2^32: 32-bit division
                        const uint32_t tile = (uint32_t)(slot >> 5);
                        trow = tile / tiles_w;
                        tcol = tile - trow * tiles_w;
                    } else {
                        const uint64_t tile = slot >> 5;
                        trow = (uint32_t)(tile / tiles_w);
                        tcol = (uint32_t)(tile - (uint64_t)trow * tiles_w);
                    }
                    const uint32_t px = tcol * kTileW + ((uint32_t)slot % kTileW);
                    const uint64_t py = (uint64_t)y0 + (uint64_t)trow * kTileH + (((uint32_t)slot & 31u) / kTileW);
                    const uint64_t i = py * cam.W + px;
                    if (px < cam.W && i >= i0 && i - i0 < n) {
                        pix = i - i0;
                        const RayIn r = pinhole_ray(cam, px, (uint32_t)py);
                        HitRec h;
                        if (w.start(f, pool, r, h)) store_hit<LAYOUT>(f, hits, pix, h);
                        else live = true;
                    }
                }
            }
            continue;
        }
        if (live) {
            for (int k = 0; k < burst; k++) {
                HitRec h;
                if (w.step(f, pool, h)) {
                    store_hit<LAYOUT>(f, hits, pix, h);
                    live = false;
                    break;
                }
            }
        }
    }
}

// Pixels i0 .. i0 + n - 1 (index px + W py); hit k of the launch is pixel i0 + k.
// Persistent variant (one launch fills the GPU; warps stay resident).  When
// at least `refill` lanes of a warp are idle, the warp takes that many new
// rays from the global queue counter `next` with one atomic and hands them to
// the idle lanes in lane order (ballot + popc rank + shuffle); busy lanes keep
// walking.  Each round advances every live lane by up to `burst` iterations.
// `next` must be zero at launch; the kernel leaves it >= n.
//
// TS: the block first copies the image's first `top_words` words (the top
// node levels of a relocated image, at most kTopSmemMaxWords) into shared
// memory, after the node stacks; the launch provides stack_bytes(J, block) +
// 4 top_words bytes of dynamic shared memory.
template <class F, int LAYOUT, int SM = 0, bool TS = false>
__global__ void __launch_bounds__(256, VX_PERSIST_MINB) k_trace_persistent(F f, const Img pool,
                                                          const float4* __restrict__ rays, uint64_t n,
                                                          void* __restrict__ hits, unsigned long long* next,
                                                          int refill, int burst, uint32_t top_words,
                                                          uint32_t sdm) {
    const unsigned lane = threadIdx.x & 31u;
    const unsigned lt_mask = (1u << lane) - 1u;
    Walker<false, F, SM, TS> w;  // node stack in the kernel's dynamic shared memory
    w.sdm = sdm;
    if (TS) {
        w.sbase_words = stack_stride((uint32_t)f.J(), 0) * blockDim.x;
        w.stw = top_words;
        uint32_t* top = reinterpret_cast<uint32_t*>(vx_dyn_smem) + 2u * w.sbase_words;
        for (uint32_t i = threadIdx.x; i < top_words; i += blockDim.x) top[i] = ldw(pool.w, i);
        __syncthreads();
    }
    bool live = false;
    bool exhausted = false;  // warp-uniform
    uint64_t idx = 0;
    while (true) {
        const unsigned idle = __ballot_sync(0xffffffffu, !live);
        if (exhausted) {
            if (idle == 0xffffffffu) break;
        } else if (__popc(idle) >= refill) {
            const int leader = __ffs(idle) - 1;
            unsigned long long base = 0;
            if ((int)lane == leader) base = atomicAdd(next, (unsigned long long)__popc(idle));
            base = __shfl_sync(0xffffffffu, base, leader);
            if (base + (unsigned long long)__popc(idle) >= n) exhausted = true;
            if (!live) {
                const uint64_t slot = base + __popc(idle & lt_mask);
                if (slot < n) {
                    idx = slot;
                    HitRec h;
                    if (w.start(f, pool, load_ray(rays, idx), h)) store_hit<LAYOUT>(f, hits, idx, h);
                    else live = true;
                }
            }
            continue;  // re-evaluate the warp's state before stepping
        }
        if (live) {
            for (int k = 0; k < burst; k++) {
                HitRec h;
                if (w.step(f, pool, h)) {
                    store_hit<LAYOUT>(f, hits, idx, h);
                    live = false;
                    break;
                }
            }
        }
    }
}

// Batched variant: the ray sets of several volumes with the same format in
// one persistent launch.  The descriptor travels in the kernel parameters;
// the queue spans the concatenated sets (set k owns slots start[k] ..
// start[k+1]-1), so warps move from set to set as sets run dry.
constexpr int kBatchMax = 64;
struct BatchDesc {
    uint32_t count;
    int packed;   // layout of every volume of the launch
    int aligned;
    const uint32_t* pool[kBatchMax];
    const float4* rays[kBatchMax];
    void* hits[kBatchMax];
    uint64_t start[kBatchMax + 1];
};

template <class F, int LAYOUT>
__global__ void __launch_bounds__(256, VX_PERSIST_MINB) k_trace_batch(F f, const __grid_constant__ BatchDesc desc,
                                                     unsigned long long* next, int refill, int burst) {
    const unsigned lane = threadIdx.x & 31u;
    const unsigned lt_mask = (1u << lane) - 1u;
    const uint64_t n = desc.start[desc.count];
    Walker<false, F> w;  // node stack in the kernel's dynamic shared memory
    bool live = false;
    bool exhausted = false;  // warp-uniform
    uint64_t idx = 0;
    int set = 0;
    // a lane's image and hit array are looked up by its set in the
    // descriptor (kernel parameters) when used, not held in registers
    auto img = [&]() { return Img{desc.pool[set], desc.packed, 0xFFFFFFFFu, desc.aligned}; };
    while (true) {
        const unsigned idle = __ballot_sync(0xffffffffu, !live);
        if (exhausted) {
            if (idle == 0xffffffffu) break;
        } else if (__popc(idle) >= refill) {
            const int leader = __ffs(idle) - 1;
            unsigned long long base = 0;
            if ((int)lane == leader) base = atomicAdd(next, (unsigned long long)__popc(idle));
            base = __shfl_sync(0xffffffffu, base, leader);
            if (base + (unsigned long long)__popc(idle) >= n) exhausted = true;
            if (!live) {
                const uint64_t slot = base + __popc(idle & lt_mask);
                if (slot < n) {
                    // the set holding this slot (binary search over the prefix)
                    int lo = 0, hi = (int)desc.count - 1;
                    while (lo < hi) {
                        const int mid = (lo + hi + 1) >> 1;
                        if (desc.start[mid] <= slot) lo = mid;
                        else hi = mid - 1;
                    }
                    set = lo;
                    idx = slot - desc.start[set];
                    HitRec h;
                    if (w.start(f, img(), load_ray(desc.rays[set], idx), h)) store_hit<LAYOUT>(f, desc.hits[set], idx, h);
                    else live = true;
                }
            }
            continue;
        }
        if (live) {
            for (int k = 0; k < burst; k++) {
                HitRec h;
                if (w.step(f, img(), h)) {
                    store_hit<LAYOUT>(f, desc.hits[set], idx, h);
                    live = false;
                    break;
                }
            }
        }
    }
}

// Up to kMaxViews camera views rendered by one launch (blockIdx.z = view):
// the views' tails overlap instead of each launch draining the GPU alone.
// View k renders its pixels [i0[k], i0[k] + n[k]) (row-major, hit index
// pixel - i0[k]) into hits[k]; y0[k] is the row of pixel i0[k].
constexpr int kMaxViews = 16;
struct ViewTable {
    CamDev cam[kMaxViews];
    void* hits[kMaxViews];
    uint64_t i0[kMaxViews], n[kMaxViews];
    uint32_t y0[kMaxViews];
};

template <class F, int LAYOUT>
__global__ void VX_PLAIN_BOUNDS k_render(F f, const Img pool, const __grid_constant__ ViewTable vt, uint32_t yoff) {
    // Each warp takes a tile of 8 x 4 pixels: neighbouring rays follow nearly
    // the same path through the format, and a compact tile has fewer lanes on
    // a silhouette than a 32-pixel run.  blockIdx.y is the tile row (image
    // rows y0 + yoff + 4 blockIdx.y ...), the x threads run along it, a warp
    // per tile, so no thread divides to find its pixel.  Pixels outside the
    // view's image or outside its [i0, i0 + n) are skipped (views of
    // different sizes share one grid).
    const int vi = (int)blockIdx.z;
    const CamDev& cam = vt.cam[vi];
    const uint32_t t = blockIdx.x * blockDim.x + threadIdx.x;
    const uint32_t lane = threadIdx.x & 31u;
    const uint32_t px = (t >> 5) * kTileW + (lane % kTileW);
    const uint64_t py = (uint64_t)vt.y0[vi] + yoff + (uint64_t)blockIdx.y * kTileH + (lane / kTileW);
    if (px >= cam.W) return;
    const uint64_t i = py * cam.W + px;
    const uint64_t i0 = vt.i0[vi];
    if (i < i0 || i - i0 >= vt.n[vi]) return;
    const RayIn r = pinhole_ray(cam, px, (uint32_t)py);
    Cnt cnt;
    const HitRec h = trace_ray<false>(f, pool, r, cnt);
    store_hit<LAYOUT>(f, vt.hits[vi], i - i0, h);
}

// ---------------------------------------------------------------------------
// Host launchers, one set per format
// ---------------------------------------------------------------------------
struct KernelSet {
    const char* spec;
    bool specialized;
    FmtParams params;
    // stack: 0 full node stack, -1 restarting traversal (Sec. 4.4), D in {1, 2, 4, 8}: short stack of depth D
    int (*trace)(const FmtParams& p, const Img pool, const float4* rays, uint64_t n,
                 void* hits, int layout, int block, int stack, cudaStream_t st);
    // count views: view k renders pixels [i0[k], i0[k] + n[k]) of cams[k] into hits[k]
    int (*render)(const FmtParams& p, const Img pool, const CamDev* cams, const uint64_t* i0, const uint64_t* n,
                  void* const* hits, int count, int layout, int block, cudaStream_t st);
    int (*trace_count)(const FmtParams& p, const Img pool, const float4* rays, uint64_t n, void* hits,
                       int layout, int block, int restart, cudaStream_t st, unsigned long long* counters,
                       uint32_t* sectors);
    int (*trace_persistent)(const FmtParams& p, const Img pool, const float4* rays,
                            uint64_t n, void* hits, int layout, int block, int blocks_per_sm, int refill, int burst,
                            int stack, uint32_t stage_words, cudaStream_t st, unsigned long long* next);
    // grid = 0: as many blocks as fit on the GPU; returns the launched grid in *grid_out.
    int (*trace_batch)(const FmtParams& p, const BatchDesc& d, int layout, int block, int grid, int refill, int burst,
                       cudaStream_t st, unsigned long long* next);
    int (*resident_blocks)(const FmtParams& p, int layout, int block, int* per_sm);
    int (*render_persistent)(const FmtParams& p, const Img pool, const CamDev& cam, uint64_t i0, uint64_t n,
                             void* hits, int layout, int block, int refill, int burst, cudaStream_t st,
                             unsigned long long* next);
};

template <class F>
struct Launch {
    static F make(const FmtParams& p);
    template <int SM>
    static int trace_as(const FmtParams& p, const Img pool, const float4* rays, uint64_t n,
                        void* hits, int layout, int block, uint32_t depth, cudaStream_t st) {
        const F f = make(p);
        const uint64_t grid = (n + (uint64_t)block - 1) / (uint64_t)block;
        const size_t sm = stack_bytes(p.J, block, depth);
        const uint32_t sdm = depth ? depth - 1u : 0u;
        prefer_carveout(layout == 0 ? (const void*)k_trace<F, 0, SM> : (const void*)k_trace<F, 1, SM>, sm, block);
        if (layout == 0) k_trace<F, 0, SM><<<(unsigned)grid, block, sm, st>>>(f, pool, rays, n, hits, sdm);
        else k_trace<F, 1, SM><<<(unsigned)grid, block, sm, st>>>(f, pool, rays, n, hits, sdm);
        return (int)cudaGetLastError();
    }
    static int trace(const FmtParams& p, const Img pool, const float4* rays, uint64_t n,
                     void* hits, int layout, int block, int stack, cudaStream_t st) {
        if (n == 0) return 0;
        if (stack < 0) return trace_as<1>(p, pool, rays, n, hits, layout, block, 0, st);
        if (stack > 0) return trace_as<2>(p, pool, rays, n, hits, layout, block, (uint32_t)stack, st);
        return trace_as<0>(p, pool, rays, n, hits, layout, block, 0, st);
    }
    static int trace_count(const FmtParams& p, const Img pool, const float4* rays, uint64_t n, void* hits,
                           int layout, int block, int restart, cudaStream_t st, unsigned long long* counters,
                           uint32_t* sectors) {
        if (n == 0) return 0;
        const F f = make(p);
        const uint64_t grid = (n + (uint64_t)block - 1) / (uint64_t)block;
        const size_t sm = stack_bytes(p.J, block);
        if (layout == 0 && !restart)
            k_trace_count<F, 0, false><<<(unsigned)grid, block, sm, st>>>(f, pool, rays, n, hits, counters, sectors);
        else if (layout == 0)
            k_trace_count<F, 0, true><<<(unsigned)grid, block, sm, st>>>(f, pool, rays, n, hits, counters, sectors);
        else if (!restart)
            k_trace_count<F, 1, false><<<(unsigned)grid, block, sm, st>>>(f, pool, rays, n, hits, counters, sectors);
        else
            k_trace_count<F, 1, true><<<(unsigned)grid, block, sm, st>>>(f, pool, rays, n, hits, counters, sectors);
        return (int)cudaGetLastError();
    }
    template <int SM, bool TS>
    static int persistent_as(const FmtParams& p, const Img pool, const float4* rays,
                             uint64_t n, void* hits, int layout, int block, int per_sm_req, int refill, int burst,
                             cudaStream_t st, unsigned long long* next, uint32_t tw, uint32_t depth = 0) {
        const F f = make(p);
        int dev = 0, sms = 0;
        cudaError_t e = cudaGetDevice(&dev);
        if (!e) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        if (e) return (int)e;
        const size_t smem = stack_bytes(p.J, block, depth) + (TS ? (size_t)tw * sizeof(uint32_t) : 0);
        const uint32_t sdm = depth ? depth - 1u : 0u;
        if (TS && smem > 48 * 1024) {  // above the default limit of dynamic shared memory
            e = layout == 0 ? cudaFuncSetAttribute(k_trace_persistent<F, 0, SM, TS>,
                                                   cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem)
                            : cudaFuncSetAttribute(k_trace_persistent<F, 1, SM, TS>,
                                                   cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
            if (e) return (int)e;
        }
        prefer_carveout(layout == 0 ? (const void*)k_trace_persistent<F, 0, SM, TS>
                                    : (const void*)k_trace_persistent<F, 1, SM, TS>,
                        smem, block);
        int per_sm = per_sm_req;
        if (per_sm <= 0) {
            e = layout == 0
                    ? cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_trace_persistent<F, 0, SM, TS>, block, smem)
                    : cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_trace_persistent<F, 1, SM, TS>, block, smem);
            if (e) return (int)e;
            if (per_sm < 1) per_sm = 1;
        }
        uint64_t grid = (uint64_t)sms * per_sm;
        const uint64_t need = (n + (uint64_t)block - 1) / (uint64_t)block;
        if (grid > need) grid = need;
        e = cudaMemsetAsync(next, 0, sizeof(unsigned long long), st);
        if (e) return (int)e;
        const unsigned g = (unsigned)grid;
        if (layout == 0)
            k_trace_persistent<F, 0, SM, TS><<<g, block, smem, st>>>(f, pool, rays, n, hits, next, refill, burst, tw,
                                                                    sdm);
        else
            k_trace_persistent<F, 1, SM, TS><<<g, block, smem, st>>>(f, pool, rays, n, hits, next, refill, burst, tw,
                                                                    sdm);
        return (int)cudaGetLastError();
    }
    // Grid = SMs x resident blocks per SM (occupancy API when blocks_per_sm is 0).
    // stage_words: stage the image's first stage_words words (at most
    // kTopSmemMaxWords; the top node levels of a relocated image) in shared
    // memory, 0 = none (not combined with restart or a short stack).
    static int trace_persistent(const FmtParams& p, const Img pool, const float4* rays,
                                uint64_t n, void* hits, int layout, int block, int blocks_per_sm, int refill,
                                int burst, int stack, uint32_t stage_words, cudaStream_t st,
                                unsigned long long* next) {
        if (n == 0) return 0;
        const uint32_t tw = stage_words <= kTopSmemMaxWords ? stage_words : 0u;
        if (stack < 0)
            return persistent_as<1, false>(p, pool, rays, n, hits, layout, block, blocks_per_sm, refill,
                                           burst, st, next, 0);
        if (stack > 0)
            return persistent_as<2, false>(p, pool, rays, n, hits, layout, block, blocks_per_sm, refill,
                                           burst, st, next, 0, (uint32_t)stack);
        if (tw)
            return persistent_as<0, true>(p, pool, rays, n, hits, layout, block, blocks_per_sm, refill,
                                          burst, st, next, tw);
        return persistent_as<0, false>(p, pool, rays, n, hits, layout, block, blocks_per_sm, refill,
                                       burst, st, next, 0);
    }
    static int resident_blocks(const FmtParams& p, int layout, int block, int* per_sm) {
        const size_t sm = stack_bytes(p.J, block);
        prefer_carveout(layout == 0 ? (const void*)k_trace_batch<F, 0> : (const void*)k_trace_batch<F, 1>, sm, block);
        cudaError_t e = layout == 0
                            ? cudaOccupancyMaxActiveBlocksPerMultiprocessor(per_sm, k_trace_batch<F, 0>, block, sm)
                            : cudaOccupancyMaxActiveBlocksPerMultiprocessor(per_sm, k_trace_batch<F, 1>, block, sm);
        if (*per_sm < 1) *per_sm = 1;
        return (int)e;
    }
    static int trace_batch(const FmtParams& p, const BatchDesc& d, int layout, int block, int grid, int refill,
                           int burst, cudaStream_t st, unsigned long long* next) {
        const F f = make(p);
        const size_t sm = stack_bytes(p.J, block);
        cudaError_t e = cudaMemsetAsync(next, 0, sizeof(unsigned long long), st);
        if (e) return (int)e;
        if (layout == 0) k_trace_batch<F, 0><<<(unsigned)grid, block, sm, st>>>(f, d, next, refill, burst);
        else k_trace_batch<F, 1><<<(unsigned)grid, block, sm, st>>>(f, d, next, refill, burst);
        return (int)cudaGetLastError();
    }
    static int render_persistent(const FmtParams& p, const Img pool, const CamDev& cam, uint64_t i0, uint64_t n,
                                 void* hits, int layout, int block, int refill, int burst, cudaStream_t st,
                                 unsigned long long* next) {
        if (n == 0) return 0;
        const F f = make(p);
        int dev = 0, sms = 0, per_sm = 1;
        const size_t sm = stack_bytes(p.J, block);
        prefer_carveout(layout == 0 ? (const void*)k_render_persistent<F, 0> : (const void*)k_render_persistent<F, 1>,
                        sm, block);
        cudaError_t e = cudaGetDevice(&dev);
        if (!e) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        if (e) return (int)e;
        e = layout == 0 ? cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_render_persistent<F, 0>, block, sm)
                        : cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_render_persistent<F, 1>, block, sm);
        if (e) return (int)e;
        if (per_sm < 1) per_sm = 1;
        // queue slots: 32 per 8 x 4 pixel tile over the rows holding pixels i0 .. i0 + n - 1
        const uint64_t y0 = i0 / cam.W, y1 = (i0 + n - 1) / cam.W;
        const uint64_t tiles_w = (cam.W + kTileW - 1) / kTileW, tile_rows = (y1 - y0 + kTileH) / kTileH;
        const uint64_t slots = tiles_w * tile_rows * 32u;
        uint64_t grid = (uint64_t)sms * per_sm;
        const uint64_t need = (slots + (uint64_t)block - 1) / (uint64_t)block;
        if (grid > need) grid = need;
        e = cudaMemsetAsync(next, 0, sizeof(unsigned long long), st);
        if (e) return (int)e;
        if (layout == 0)
            k_render_persistent<F, 0><<<(unsigned)grid, block, sm, st>>>(f, pool, cam, i0, n, (uint32_t)y0,
                                                                         (uint32_t)tiles_w, slots, hits, next,
                                                                         refill, burst);
        else
            k_render_persistent<F, 1><<<(unsigned)grid, block, sm, st>>>(f, pool, cam, i0, n, (uint32_t)y0,
                                                                         (uint32_t)tiles_w, slots, hits, next,
                                                                         refill, burst);
        return (int)cudaGetLastError();
    }
    static int render(const FmtParams& p, const Img pool, const CamDev* cams, const uint64_t* i0, const uint64_t* n,
                      void* const* hits, int count, int layout, int block, cudaStream_t st) {
        const F f = make(p);
        const size_t sm = stack_bytes(p.J, block);
        prefer_carveout(layout == 0 ? (const void*)k_render<F, 0> : (const void*)k_render<F, 1>, sm, block);
        constexpr uint64_t kMaxRows = 65535;
        // launches of up to kMaxViews views; 8 x 4 pixel tiles over the image
        // rows that hold each view's pixels; one grid row per tile row (the
        // views' largest count, at most 65535 per launch), one grid column
        // block per `block` threads of the widest view's tile row
        for (int v0 = 0; v0 < count; v0 += kMaxViews) {
            ViewTable vt{};
            int nv = 0;
            uint64_t rows = 0, row_threads = 0;
            for (int k = v0; k < count && k < v0 + kMaxViews; k++) {
                if (n[k] == 0) continue;
                const CamDev& cam = cams[k];
                const uint64_t y0 = i0[k] / cam.W, y1 = (i0[k] + n[k] - 1) / cam.W;
                const uint64_t tiles_w = (cam.W + kTileW - 1) / kTileW;
                const uint64_t tile_rows = (y1 - y0 + kTileH) / kTileH;
                if (tile_rows > rows) rows = tile_rows;
                if (tiles_w * 32u > row_threads) row_threads = tiles_w * 32u;
                vt.cam[nv] = cam;
                vt.hits[nv] = hits[k];
                vt.i0[nv] = i0[k];
                vt.n[nv] = n[k];
                vt.y0[nv] = (uint32_t)y0;
                nv++;
            }
            if (nv == 0) continue;
            if (row_threads + (uint64_t)block > 0xFFFFFFFFull) return (int)cudaErrorInvalidConfiguration;
            const unsigned gx = (unsigned)((row_threads + (uint64_t)block - 1) / (uint64_t)block);
            for (uint64_t r = 0; r < rows; r += kMaxRows) {
                const dim3 grid(gx, (unsigned)(rows - r < kMaxRows ? rows - r : kMaxRows), (unsigned)nv);
                const uint32_t yoff = (uint32_t)(r * kTileH);
                if (layout == 0)
                    k_render<F, 0><<<grid, block, sm, st>>>(f, pool, vt, yoff);
                else
                    k_render<F, 1><<<grid, block, sm, st>>>(f, pool, vt, yoff);
            }
            const cudaError_t e = cudaGetLastError();
            if (e) return (int)e;
        }
        return 0;
    }
};

template <>
inline DynF Launch<DynF>::make(const FmtParams& p) {
    DynF f;
    f.p = p;
    return f;
}
template <class F>
inline F Launch<F>::make(const FmtParams&) {
    return F{};
}

template <class Fm>
KernelSet make_kernel_set(const char* spec) {
    using F = typename Fm::F;
    return KernelSet{spec, true, Fm::P, &Launch<F>::trace, &Launch<F>::render, &Launch<F>::trace_count,
                     &Launch<F>::trace_persistent, &Launch<F>::trace_batch, &Launch<F>::resident_blocks,
                     &Launch<F>::render_persistent};
}

void register_kernel_set(const KernelSet* ks);

struct KernelSetRegistrar {
    explicit KernelSetRegistrar(const KernelSet* ks) { register_kernel_set(ks); }
};

}  // namespace vx
