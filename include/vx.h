/*
 * vx.h -- C ABI of libvx: hybrid voxel formats (Arbore et al., "Hybrid Voxel
 * Formats for Efficient Ray Tracing") built on the host and traced on an
 * NVIDIA B300 (sm_103a).
 *
 * A hybrid format is a list of levels, each one of the paper's base formats
 * (Sec. 3.1, Table 1): Raw R(W,H,D), distance field D(W,H,D,M), SVO S(L) or
 * SVDAG G(L).  A voxel holds a 32-bit RGBA word (R | G << 8 | B << 16 |
 * A << 24) and is empty iff all 32 bits are 0 (Sec. 3).  The library builds a volume in the paper's word-buffer
 * layout (Sec. 3.3, Fig. 3) with the Morton-order construction of Sec. 4.1 and
 * Sec. 5, copies it to the GPU, and answers first-hit ray queries with CUDA
 * kernels whose per-level steppers are composed at compile time (Sec. 4.2).
 *
 * Conventions shared by every call:
 *   - return value 0 (VX_OK) or a negative VX_E* code; on error,
 *     vx_last_error() returns a message for the calling thread;
 *   - device pointers are plain CUDA device addresses owned by the caller;
 *     host pointers are plain host addresses owned by the caller; a call never
 *     frees memory it did not allocate;
 *   - `stream` is a cudaStream_t (NULL = the legacy default stream); calls
 *     that take one enqueue work on it and return without synchronising,
 *     except the *_host variants, which return when their results are in host
 *     memory;
 *   - all calls are thread-safe for distinct volumes; a volume may be traced
 *     from several threads/streams at once, but must not be freed while in use.
 */
#ifndef VX_H_
#define VX_H_

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ----------------------------------------------------------------------- */
/* Error codes                                                              */
/* ----------------------------------------------------------------------- */
#define VX_OK 0
#define VX_EINVAL (-1)       /* bad argument, bad format spec, misaligned pointer */
#define VX_ENOMEM (-2)       /* host or device allocation failed */
#define VX_ECUDA (-3)        /* a CUDA call failed (message names it) */
#define VX_ETOOBIG (-4)      /* buffer would exceed 2^32 words (Sec. 3.3) */
#define VX_ETIMEOUT (-5)     /* a bounded device wait ran out */
#define VX_EUNSUPPORTED (-6) /* valid request this build cannot serve */

/* ----------------------------------------------------------------------- */
/* Rays and hits                                                            */
/* ----------------------------------------------------------------------- */
/* One ray, 32 bytes, 16-byte aligned in arrays: points o + t d for
 * t in [tmin, tmax], in voxel units over the box [0,nx) x [0,ny) x [0,nz).
 * d need not be normalised.  A ray with a NaN component or an infinite tmin
 * is reported with status VX_STATUS_INVALID. */
typedef struct vx_ray {
    float ox, oy, oz, tmin;
    float dx, dy, dz, tmax;
} vx_ray;

/* Full hit record, 16 bytes (hit_layout = VX_HIT_FULL).
 *   t      entry parameter of the hit voxel (tmin / box entry for the first
 *          voxel); +inf on a miss;
 *   rgba   the voxel's word; 0 on a miss;
 *   x,y,z  voxel coordinate; 0xFFFF on a miss;
 *   face   0 = ray starts inside the voxel, else 1 + 2*axis + (d_axis < 0):
 *          the side the ray entered through;
 *   status VX_STATUS_*. */
typedef struct vx_hit {
    float t;
    uint32_t rgba;
    uint16_t x, y, z;
    uint8_t face;
    uint8_t status;
} vx_hit;

/* Compact hit record, 8 bytes (hit_layout = VX_HIT_COMPACT): idx =
 * x + nx*(y + ny*z), or 0xFFFFFFFF for a miss or an invalid ray; t as above.
 * Needs nx*ny*nz < 2^32. */
typedef struct vx_hit_compact {
    uint32_t idx;
    float t;
} vx_hit_compact;

#define VX_HIT_FULL 0
#define VX_HIT_COMPACT 1

#define VX_STATUS_MISS 0
#define VX_STATUS_HIT 1
#define VX_STATUS_INVALID 2
#define VX_STATUS_ERROR 3 /* iteration cap or bounds check tripped */

/* ----------------------------------------------------------------------- */
/* Volumes                                                                  */
/* ----------------------------------------------------------------------- */
typedef struct vx_volume_s* vx_volume;

/* Source grid of a build, the role of the paper's voxelizer (Sec. 4.1,
 * Sec. 5).  Exactly one of `dense`, `dense_pal` and `fill_brick` is set.
 *   log2_dim  grid size per axis, 2^log2_dim[i] voxels (<= 2^15);
 *   dense     host array of 2^(sum log2_dim) RGBA words, x fastest;
 *   dense_pal host array of 2^(sum log2_dim) 8-bit palette indices, x
 *             fastest, with `palette` (256 RGBA words, palette[0] = 0);
 *   fill_brick  called with a cube of side 2^log2_size whose corner
 *             (x0,y0,z0) is a multiple of its side; writes the cube's words,
 *             x fastest, to `out`; returns 0 on success;
 *   block_empty optional: returns 1 only if the cube holds no occupied voxel
 *             (lets the builder skip empty space without fetching it);
 *   user      passed back to the callbacks. */
typedef int (*vx_fill_brick_fn)(void* user, uint32_t x0, uint32_t y0, uint32_t z0, uint32_t log2_size,
                                uint32_t* out);
typedef int (*vx_block_empty_fn)(void* user, uint32_t x0, uint32_t y0, uint32_t z0, uint32_t log2_size);
typedef struct vx_grid {
    uint32_t log2_dim[3];
    const uint32_t* dense;
    vx_fill_brick_fn fill_brick;
    vx_block_empty_fn block_empty;
    void* user;
    const uint8_t* dense_pal;
    const uint32_t* palette;
} vx_grid;

#define VX_DEDUP_PER_SUBVOLUME 0
#define VX_DEDUP_WHOLE_LEVEL 1 /* the paper's evaluated setting (Sec. 6.1) */

/* Build options (NULL = defaults).
 *   dedup_scope   VX_DEDUP_WHOLE_LEVEL (default) or VX_DEDUP_PER_SUBVOLUME:
 *                 one SVDAG de-duplication map per level, or one per
 *                 sub-volume (Sec. 4.3);
 *   device        CUDA device for the device image; -1 = current (default);
 *   no_upload     1 = build on the host only (vx_trace then fails);
 *   threads       host threads for the build, 0 = all cores;
 *   canonical_device  1 = put the canonical words on the device as they
 *                 are; 0 (default) = a device image with the same structures
 *                 in the same order, relocated so that every DF cell array,
 *                 SVO root entry and SVO child list starts at an even word
 *                 (a DF cell {terminating integer, distance} and an SVO node
 *                 entry {pointer, masks} are then one 8-byte load; one zero
 *                 word of padding where needed), and, when the format has an
 *                 SVDAG level and the image stays below 2^24 words, packed:
 *                 each pointer to an SVDAG node carries the node's valid mask
 *                 in bits 24..31 and an SVDAG slot of a leaf child holds the
 *                 leaf's terminating integer (the leaf words are dropped),
 *                 which saves one or two dependent reads per SVDAG level.
 *                 vx_canonical always returns the paper's layout; vx_stats
 *                 reports the device image's size and which changes apply;
 *   generic_kernel  1 = trace with the kernels that take the format as a
 *                 run-time argument even when a compile-time-composed kernel
 *                 exists for the spec (same results; for checking the two
 *                 against each other); 0 (default) = the compile-time kernel
 *                 when one is compiled in (see vx_formats). */
typedef struct vx_build_opts {
    int32_t dedup_scope;
    int32_t device;
    int32_t no_upload;
    int32_t threads;
    int32_t canonical_device;
    int32_t generic_kernel;
    int32_t reserved[2];
} vx_build_opts;

/* Builds `spec` over `grid` and uploads it.  Paper: Sec. 4.1 (per-level
 * construction, Fig. 4 construct), Sec. 5 (Morton order), Sec. 3.3 (layout).
 *   spec  format signature in Table 1's grammar with log2 extents, levels
 *         separated by spaces: "R(4,4,4) S(2) G(3)"; "R(4^3)" abbreviates
 *         R(4,4,4).  Each level but the first must be cubic (Sec. 5); the
 *         extents per axis must sum to grid->log2_dim.
 *   out   receives the handle; free it with vx_free.
 * Errors: VX_EINVAL (spec or grid), VX_ETOOBIG (over 2^32 words, Sec. 3.3),
 * VX_ENOMEM, VX_ECUDA, VX_EUNSUPPORTED (a level kind this build lacks). */
int vx_build(const char* spec, const vx_grid* grid, const vx_build_opts* opts, vx_volume* out);

/* Signatures of the formats whose kernels are composed at compile time
 * (Sec. 4: the paper generates one intersection function per level of a
 * format; here C++ templates fold each listed format into constants).  Any
 * other valid signature is traced by the kernels that read the format as a
 * run-time argument.
 *   specs     NULL, or an array of `capacity` pointers that receives the
 *             first min(capacity, count) signatures, in the canonical
 *             spelling vx_build accepts (static strings, never freed);
 *   count     receives the number of compiled-in formats.
 * Errors: VX_EINVAL (count NULL). */
int vx_formats(const char** specs, uint32_t capacity, uint32_t* count);

/* Releases the host and device memory of a volume (synchronises its device
 * first).  NULL is accepted. */
int vx_free(vx_volume v);

/* A volume from a word buffer in the paper's layout (Sec. 3.3) -- e.g. one
 * saved from vx_canonical -- for format `spec`; n_words >= 1, word 0 the root
 * pointer.  The words are copied.  validate != 0 (the normal case) walks the
 * whole buffer first: every pointer inside the buffer, octree masks
 * consistent with their depth (leaf mask set exactly at the last depth),
 * non-empty valid children, every DF distance equal to its definition;
 * failure is VX_EINVAL with the offending word in vx_last_error().
 * validate == 0 skips the walk and marks the volume unvalidated: every trace
 * entry point then refuses it (VX_EINVAL) except vx_trace_counted, whose
 * reads are checked.  opts as for vx_build (dedup_scope and threads unused).
 * Stats: canonical_words and per-level words / node counts (from the walk),
 * occupied_voxels 0.  Errors: VX_EINVAL (spec, empty or malformed buffer),
 * VX_ETOOBIG (n_words >= 2^32, checked before any word is read), VX_ENOMEM,
 * VX_ECUDA.  The paper has no loader: its construction writes the buffer to
 * a file (Sec. 4.1); this reads such a buffer back. */
int vx_load(const char* spec, const uint32_t* words, uint64_t n_words, const vx_build_opts* opts, int32_t validate,
            vx_volume* out);

/* Host view of the canonical (paper-layout) word buffer: word 0 is the root
 * pointer (Sec. 4.1).  The pointer stays valid until vx_free. */
int vx_canonical(vx_volume v, const uint32_t** words, uint64_t* n_words);

/* Decodes the voxels of an axis-aligned cube of side 2^log2_size at
 * (x0,y0,z0) (a multiple of the side) from the canonical buffer into `out`
 * (host, x fastest).  Host only; for checks and tools. */
int vx_decode_brick(vx_volume v, uint32_t x0, uint32_t y0, uint32_t z0, uint32_t log2_size, uint32_t* out);

/* ----------------------------------------------------------------------- */
/* Tracing                                                                  */
/* ----------------------------------------------------------------------- */
#define VX_MODE_AUTO 0       /* pick per format (autotuned when tuned) */
#define VX_MODE_PLAIN 1      /* one thread per ray */
#define VX_MODE_PERSISTENT 2 /* persistent warps refilled from a global ray queue */

/* Trace options (NULL = defaults / autotuned values).
 *   mode   VX_MODE_*;
 *   block  threads per block: 0 = default (256 for persistent kernels, 64
 *          for the plain trace kernel, 128 for the plain render kernel),
 *          else a multiple of 32 in [32, 256] (VX_EINVAL otherwise);
 *   blocks_per_sm  persistent mode: resident blocks per SM, 0 = as many as fit;
 *   smem_top  persistent mode, staging depth: k in [1, 8] = each block first
 *          copies the structures of the top k node levels (any level kind:
 *          Raw, DF, SVO, SVDAG) into shared memory and reads them there; the
 *          device image holds them as one prefix, level by level.  The
 *          largest depth <= k whose prefix fits 8192 words (32 KiB) is used;
 *          none for a canonical device image, with restart or with a short
 *          stack.  0 = off.  Any other value: VX_EINVAL;
 *   refill persistent mode: a warp fetches new rays once this many of its
 *          lanes are idle (1..32), 0 = default;
 *   burst  persistent mode: loop iterations between refill checks, 0 = default;
 *   sort_cell_log2  0 = trace rays in the given order; g in [1, 15] = first
 *          sort them by (direction octant, Morton code of the origin's cell of
 *          side 2^g) for coherence; hits still land in the caller's order.
 *          The sort copies the rays into key order, the trace writes hits
 *          in that order and a gather puts each back at its ray's index, so
 *          the trace reads and writes whole sectors in order.  Sorting takes
 *          40 B per ray plus one hit record per ray, plus at most 1 MiB +
 *          384 B, of device scratch from CUDA's stream-ordered allocator
 *          (cudaMallocAsync), at most 2^32 - 1 rays per call;
 *   restart 0 = octree levels keep a per-ray stack of the nodes entered;
 *          1 = restarting sparse-voxel intersection (Sec. 4.4): keep only
 *          each format level's root and walk an SVO / SVDAG level again from
 *          its root after leaving one of its nodes (same results, no stack
 *          per octree depth, redundant node reads).  Used by vx_trace and
 *          vx_trace_counted; vx_render, vx_trace_batch and vx_trace_noalloc
 *          always keep the stack.  Any other value: VX_EINVAL;
 *   short_stack 0 = the full node stack (one entry per node level); D in
 *          {1, 2, 4, 8} = keep each format level's root node and, for the
 *          octree levels below it, only a ring of the D most recently entered
 *          nodes: leaving a node whose ancestor fell out of the ring walks
 *          that format level again from its root (the restart of Sec. 4.4),
 *          so results are the same with less per-ray state.  Used by vx_trace
 *          (plain and persistent; not with smem_top, which it turns off).
 *          VX_EINVAL for other values or together with restart = 1.
 * Persistent launches (and the kernels of vx_trace_batch) each need a
 * ray-queue counter of the volume.  A launch issued directly takes one from a
 * ring of 256 per volume, so at most 256 of them may be in flight at once per
 * volume.  A launch captured into a CUDA graph gets a counter of its own,
 * which every replay of that graph reuses and no other launch ever takes; a
 * volume has 3840 of those, and a capture beyond them fails with
 * VX_EUNSUPPORTED.  Replays of one graph must therefore not overlap each
 * other (replay it on one stream). */
typedef struct vx_trace_opts {
    int32_t mode;
    int32_t block;
    int32_t blocks_per_sm;
    int32_t smem_top;
    int32_t refill;
    int32_t burst;
    int32_t sort_cell_log2;
    int32_t restart;
    int32_t short_stack;
} vx_trace_opts;

/* Size and build statistics of a volume.  Level k counts the words written
 * for its structures (Raw arrays, octree node lists, DAG nodes) and its
 * nodes: Raw sub-volumes, or octree / DAG nodes including leaf nodes. */
#define VX_MAX_LEVELS 16
typedef struct vx_stats {
    uint32_t n_levels;
    uint32_t n_node_levels;  /* levels after expanding S(L)/G(L) into L octree levels */
    uint32_t log2_dim[3];
    int32_t specialized;     /* 1 = a compile-time-composed kernel serves this spec */
    int32_t packed;          /* 1 = the device image uses the packed layout */
    int32_t aligned;         /* 1 = the device image is relocated with two-word structures at even words */
    uint64_t canonical_words;   /* paper-layout buffer size in words */
    uint64_t device_bytes;      /* device image size */
    uint64_t occupied_voxels;
    uint64_t level_words[VX_MAX_LEVELS];
    uint64_t level_nodes[VX_MAX_LEVELS];
    double build_ms;
    double upload_ms;
    int32_t tuned;              /* 1 once vx_autotune has chosen options */
    vx_trace_opts tuned_opts;   /* the options VX_MODE_AUTO traces use (valid when tuned) */
} vx_stats;

int vx_stats_get(vx_volume v, vx_stats* out);

/* First hit of each ray (Sec. 4.2: the root function reads the root pointer,
 * tests the root box and calls the level functions, which visit non-empty
 * sub-volumes in hit-time order, Fig. 4 intersect).
 *   rays  device array of n vx_ray (16-byte aligned);
 *   hits  device array of n vx_hit or vx_hit_compact (per hit_layout),
 *         16- or 8-byte aligned;
 * Results equal a plain FP64 Amanatides-Woo walk over the uncompressed grid.
 * Errors: VX_EINVAL (NULL or misaligned pointers, bad layout, compact layout
 * on a grid of 2^32 voxels or more), VX_ECUDA (launch failure). */
int vx_trace(vx_volume v, const vx_ray* rays, uint64_t n, void* hits, int32_t hit_layout,
             const vx_trace_opts* opts, void* stream);

/* Same results as vx_trace from an instrumented kernel that also adds, over
 * all rays, into the device array counters[0..3] (caller-zeroed, 8-byte
 * aligned, unsigned 64-bit): [0] bytes of the format read by the traversal
 * (Raw cell 4, DF cell 8, octree node 8, DAG mask 4 + pointer 4, leaf
 * terminating integer 4), [1] loop iterations, [2] decisions re-taken in
 * FP64, [3] reads refused because they fell outside the volume's words.
 * For measurement: the bytes a ray must read from the format are the
 * algorithmic traffic of the method.  This kernel checks every read of the
 * volume against its size: a refused read counts in [3] and the ray's hit
 * reports VX_STATUS_ERROR, so it is the one trace that may read a volume
 * loaded without validation (vx_load).
 *   sectors  NULL, or a caller-zeroed device array of
 *            ceil(device_bytes / 1024) uint32 words (4-byte aligned; see
 *            vx_stats): bit (s & 31) of word s >> 5 is set when the traversal
 *            read any word of the s-th 32-byte sector of the device image.
 *            Its popcount x 32 B is the format's footprint in the launch, the
 *            bytes a cold cache must fetch from DRAM at least.  Bits are only
 *            ever set (atomic OR), so calls may accumulate into one array. */
int vx_trace_counted(vx_volume v, const vx_ray* rays, uint64_t n, void* hits, int32_t hit_layout,
                     const vx_trace_opts* opts, void* stream, unsigned long long* counters, uint32_t* sectors);

/* Several ray sets, possibly through different volumes (all on one device),
 * in one call: the sets are grouped by format, each group (up to 64 sets) is
 * traced by one persistent kernel whose warps take rays from a queue that
 * spans all of the group's sets, and the groups' kernels are enqueued on
 * forked streams, each with a full GPU's worth of blocks, so that one
 * group's blocks start as the previous group's retire.  Hits of set k
 * land in items[k].hits in the set's own order, exactly as vx_trace would
 * write them.  The call enqueues work on `stream` and returns; it allocates
 * nothing and does not synchronise, so it can be captured into a CUDA graph
 * (make one uncaptured call per device first: it creates the library's
 * fork streams).  opts: refill/burst/block as for vx_trace for every group
 * (NULL or VX_MODE_AUTO: the options vx_autotune_batch chose for each
 * group's volume, else block 256, refill 4, burst 16 for every group; the
 * options vx_autotune picks for vx_trace are not used here); sorting is not
 * supported
 * here (VX_EUNSUPPORTED).  Calls for one device are enqueued one at a time.
 * (Not in the paper: it traces one frame of one format at a time.) */
typedef struct vx_batch_item {
    vx_volume volume;
    const vx_ray* rays; /* device, 16-byte aligned */
    uint64_t n;
    void* hits;         /* device, per hit_layout */
} vx_batch_item;
int vx_trace_batch(const vx_batch_item* items, uint32_t count, int32_t hit_layout, const vx_trace_opts* opts,
                   void* stream);

/* vx_trace_batch that also times its kernels: it records caller-created
 * CUDA events (cudaEvent_t, created with timing enabled) on the stream each
 * group's kernel runs on, events[2k] just before group k's kernel and
 * events[2k + 1] just after it, so cudaEventElapsedTime of the pair is that
 * kernel's duration.  Groups are numbered in the order their first set
 * appears in `items` (a format with more than 64 sets forms several groups,
 * consecutive); groups k >= n_events / 2 are not timed.  *groups (optional)
 * receives the number of groups launched.  Capturable like vx_trace_batch
 * (the records become event nodes of the graph).  Errors as vx_trace_batch,
 * plus VX_EINVAL for n_events > 0 with events NULL. */
int vx_trace_batch_timed(const vx_batch_item* items, uint32_t count, int32_t hit_layout, const vx_trace_opts* opts,
                         void* stream, void** events, uint32_t n_events, uint32_t* groups);

/* vx_trace_batch for rays and hits in host memory (items[k].rays and
 * .hits are host pointers, aligned as for vx_trace_batch; page-locked memory
 * gives full-speed asynchronous copies, pageable memory works but its copies
 * do not overlap).  The rays of all items stream through the device in waves
 * of at most 2^21 rays, taken in item order (an item larger than the room
 * left in a wave is split across waves); each wave is uploaded, traced by
 * the batched kernels (as vx_trace_batch: one persistent kernel per format,
 * each volume's batched options unless opts is given) and its hits copied
 * back, with four waves in flight on four internal streams, so uploads,
 * kernels and downloads overlap.  The first wave starts after the caller's
 * earlier work on `stream`; the call returns when every hit is in host
 * memory.  Device scratch: four wave buffers of 96 MiB, allocated on the
 * first call per device and kept for the process; calls on one device run
 * one at a time.  Errors as vx_trace_batch, and VX_EUNSUPPORTED when
 * `stream` is being captured into a CUDA graph (the call waits for its
 * copies); on an error the call still waits for the copies it issued
 * before returning. */
int vx_trace_batch_host(const vx_batch_item* items, uint32_t count, int32_t hit_layout, const vx_trace_opts* opts,
                        void* stream);

/* Picks the batched kernel's options for each volume among the items.  The
 * objective is the whole call (the groups' kernels run concurrently and
 * share the SMs): coordinate descent over the refill threshold (1-16),
 * iterations per refill check (4-32) and block size (128, 256), first for
 * all volumes together (two rounds), then for each volume with the others
 * fixed (one round), each candidate timed as the vx_trace_batch call over
 * all items on `stream` (best of three after one warm-up call; a candidate
 * replaces the current options only when more than 1% faster), starting
 * from the options a batched call would use now.  Later vx_trace_batch,
 * vx_trace_batch_timed and vx_trace_batch_host calls with opts NULL or
 * VX_MODE_AUTO use them for each volume's group.  Traces every item many
 * times (hits are overwritten with the same records); synchronises
 * `stream`.  chosen (optional, count entries) receives, per item, its
 * volume's options (zeros for a volume with no rays in the items).  Errors
 * as vx_trace_batch.  (Not in the paper.) */
int vx_autotune_batch(const vx_batch_item* items, uint32_t count, int32_t hit_layout, void* stream,
                      vx_trace_opts* chosen);

/* Picks vx_trace options for this volume: times candidates on `rays` (a
 * device sample of the rays the caller will trace, n of them) with CUDA
 * events on `stream` (each candidate the best of three launches) --
 * restarting vs stack traversal, short-stack depth, shared-memory staging
 * depth, coherence-sort granularity, persistent refill threshold,
 * iterations per refill check, block size (two rounds), then the plain
 * kernel at each block size -- by coordinate descent (a candidate replaces
 * the current options only when more than 1% faster), and keeps the
 * result; later vx_trace calls with
 * opts NULL or mode VX_MODE_AUTO use it.  Synchronises `stream`; allocates a
 * temporary n-hit buffer.  best (optional) receives the options, best_ms the
 * sample's time with them.  (Not in the paper: its formats are traced with
 * one fixed GLSL shader per format.) */
int vx_autotune(vx_volume v, const vx_ray* rays, uint64_t n, void* stream, vx_trace_opts* best, double* best_ms);

/* Same as vx_trace with host arrays: the rays are copied to the device in
 * chunks, traced and the hits copied back, copies overlapped with tracing.
 * Returns when all hits are in host memory.  Pinned host memory is fastest.
 * VX_EUNSUPPORTED on a stream being captured into a CUDA graph (as for
 * vx_render_host). */
int vx_trace_host(vx_volume v, const vx_ray* rays_host, uint64_t n, void* hits_host, int32_t hit_layout,
                  const vx_trace_opts* opts, void* stream);

/* vx_trace for callers that cannot allocate device memory while tracing:
 * applications whose own allocator owns the GPU's memory, real-time loops
 * that forbid allocation (and the synchronisation it implies) after start-up,
 * plug-ins whose host manages device memory.  The paper has no counterpart;
 * this is a service of the library.
 * Same hits as vx_trace (the persistent kernel, format described at run time).
 * Its only scratch, a 32-bit ray-queue counter, sits in a 256-byte static
 * device array that every GPU which loads the library keeps until the process
 * exits; the call itself never calls cudaMalloc or cudaFree.
 *   - The first call on a device looks up the array's device address
 *     (cudaGetSymbolAddress) with that device current: make that first call
 *     before any stream capture.  The address is kept for the process; it
 *     stays valid until the device's primary context is destroyed
 *     (cudaDeviceReset), after which this entry point must not be called.
 *   - All calls share the array; each zeroes the counter on its stream before
 *     its launch, so calls whose kernels overlap on the GPU race: issue them
 *     one after another (e.g. on one stream).
 *   - n must not exceed VX_NOALLOC_MAX_RAYS (VX_EINVAL otherwise).
 * Arguments and errors otherwise as vx_trace (block size and mode fixed). */
#define VX_NOALLOC_MAX_RAYS 4278190080ull /* 2^32 - 2^24 */
int vx_trace_noalloc(vx_volume v, const vx_ray* rays, uint64_t n, void* hits, int32_t hit_layout, void* stream);

/* ----------------------------------------------------------------------- */
/* Ray generation                                                           */
/* ----------------------------------------------------------------------- */
/* Pinhole camera: pixel (px, py), py = 0 at the top row, gets the ray through
 * its centre: d = normalize(f + sx r + sy u) with f = normalize(look - eye),
 * r = normalize(f x up), u = r x f, sx = (2 (px + 0.5)/W - 1) tan(vfov/2) W/H,
 * sy = (1 - 2 (py + 0.5)/H) tan(vfov/2); origin eye, tmin 0, tmax +inf.
 * Ray index px + W py.  (The paper renders camera views, Fig. 6; it fixes no
 * camera model.) */
typedef struct vx_camera {
    double eye[3], look[3], up[3];
    double vfov_deg;
    uint32_t width, height;
} vx_camera;

/* Writes width*height rays to `rays` (device, 16-byte aligned). */
int vx_raygen_pinhole(const vx_camera* cam, vx_ray* rays, void* stream);

/* Ambient-occlusion rays from n primary rays and their full hit records
 * (device): spp rays per primary, index i * spp + k, cosine-weighted about
 * the outward normal of the face the primary ray entered (Malley's method:
 * uniform point on the unit disk, r = sqrt(u1), phi = 2 pi u2, lifted by
 * z = sqrt(1 - u1)); tangents e_{a+1}, e_{a+2} (mod 3) for normal axis a.
 * u1, u2 = top 24 bits of SplitMix64(SplitMix64(seed) ^ c), c = (i * spp +
 * k) * 2 and c + 1 (Steele, Lea & Flood 2014).  Origin = o + t d of the
 * primary, moved eps along the normal; tmin 0, tmax `tmax`.  Misses and
 * hits with face 0 give the all-zero ray (traced as a miss).  The paper
 * evaluates without shading from bounces (Fig. 5 caption); this is the
 * secondary-ray workload of the benchmark. */
int vx_raygen_ao(const vx_ray* rays, const void* hits, uint64_t n, uint64_t seed, uint32_t spp, float eps, float tmax,
                 vx_ray* out, void* stream);

/* Pinhole rays generated and traced in one kernel (no ray array in memory);
 * hits as for vx_trace, one per pixel (hit x + width * y belongs to pixel
 * (x, y)).  opts: mode VX_MODE_PLAIN (one thread per pixel, each warp an
 * 8 x 4 pixel tile, blocks of 128 by default; the default mode, also for
 * NULL / AUTO) or VX_MODE_PERSISTENT (pixels taken in row order from a queue
 * by persistent warps); refill, burst, block as for vx_trace (the volume's
 * tuned options are not used here). */
int vx_render(vx_volume v, const vx_camera* cam, void* hits, int32_t hit_layout, const vx_trace_opts* opts,
              void* stream);

/* Several camera views of one volume in one call: view k renders cams[k]
 * into hits[k] (device, per hit_layout, one record per pixel as for
 * vx_render).  In plain mode (the default) up to 16 views share one launch
 * (one grid layer per view, the tiles of all views in flight together), so
 * the views' last warps overlap instead of each view draining the GPU
 * alone; results are those of one vx_render per view.  VX_MODE_PERSISTENT
 * renders one view per launch.  Errors as vx_render, naming the view. */
int vx_render_views(vx_volume v, const vx_camera* cams, uint32_t count, void* const* hits, int32_t hit_layout,
                    const vx_trace_opts* opts, void* stream);

/* Same as vx_render with the hits copied to host memory; returns when they
 * are there.  VX_EUNSUPPORTED on a stream being captured into a CUDA graph. */
int vx_render_host(vx_volume v, const vx_camera* cam, void* hits_host, int32_t hit_layout,
                   const vx_trace_opts* opts, void* stream);

/* ----------------------------------------------------------------------- */
/* Misc                                                                     */
/* ----------------------------------------------------------------------- */
/* Message of the last failed call on this thread ("" if none). */
const char* vx_last_error(void);

/* Library version, major * 10000 + minor * 100 + patch. */
int vx_version(void);

#ifdef __cplusplus
}
#endif
#endif /* VX_H_ */
