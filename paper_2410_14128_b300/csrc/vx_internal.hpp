// vx_internal.hpp -- host-side declarations shared by the library's
// translation units (not part of the public C ABI).
#pragma once
#include <stdint.h>

#include <atomic>
#include <memory>
#include <mutex>
#include <string>
#include <vector>

#include "../../include/vx.h"
#include "fmt.hpp"

namespace vx {

// ---------------------------------------------------------------------------
// Errors: thread-local message returned by vx_last_error().
// ---------------------------------------------------------------------------
int fail(int code, const char* fmt, ...);
void clear_error();

// ---------------------------------------------------------------------------
// Format signatures (Table 1 grammar, log2 extents).
// ---------------------------------------------------------------------------
struct Level {
    int kind;  // Kind
    int e[3];  // Raw / DF: W,H,D; SVO/SVDAG: L,L,L
    int m;     // DF: distance cap M
};

constexpr int kMaxDfCap = 65535;  // largest DF distance cap M (also bounds every number in a spec)

struct Spec {
    std::vector<Level> lv;
    int ldim[3] = {0, 0, 0};
    FmtParams fmt{};
    std::string canonical;  // normalised text, e.g. "R(4,4,4) S(2) G(3)"
};

// Parses and validates a signature.  Returns VX_OK or a VX_E* code.
int parse_spec(const char* text, Spec* out);

// Morton order (x lowest bit, Fig. 5); extents may differ per axis: bits are
// interleaved x, y, z while each axis still has bits left.
void morton_decode(uint64_t m, const int e[3], uint32_t c[3]);
uint64_t morton_encode(const uint32_t c[3], const int e[3]);

// ---------------------------------------------------------------------------
// Voxel sources (the voxelizer role of Sec. 4.1).
// ---------------------------------------------------------------------------
class VoxelSource {
  public:
    virtual ~VoxelSource() {}
    // True when concurrent calls are safe (the parallel build needs it).
    virtual bool thread_safe() const { return false; }
    // True only if the cube of side 2^log2s at (x0,y0,z0) holds no occupied voxel.
    virtual bool empty(int64_t x0, int64_t y0, int64_t z0, int log2s) = 0;
    // Words of the cube (side 2^log2s, corner a multiple of the side), x fastest.
    virtual int block(int64_t x0, int64_t y0, int64_t z0, int log2s, uint32_t* out) = 0;
};

VoxelSource* make_dense_source(const uint32_t* words, const int ldim[3]);
VoxelSource* make_brick_source(const vx_grid* g);
VoxelSource* make_palette_source(const uint8_t* idx, const uint32_t* palette, const int ldim[3]);

// ---------------------------------------------------------------------------
// Canonical build (paper layout) and its statistics.
// ---------------------------------------------------------------------------
struct BuildResult {
    std::vector<uint32_t> words;  // word 0 = root pointer
    uint64_t level_words[VX_MAX_LEVELS] = {};
    uint64_t level_nodes[VX_MAX_LEVELS] = {};
    uint64_t occupied = 0;
};

// threads: 1 = sequential; 0 = all cores; the parallel path needs a Raw or DF
// top level and a thread-safe source, and gives the same words as the sequential.
int build_canonical(const Spec& spec, VoxelSource& src, int dedup_scope, BuildResult* out, int threads);

// L1 distance of every cell of a W x H x D grid (terms != 0 are non-empty) to
// the nearest non-empty cell, capped at M (the DF level of Table 1).
void l1_distance(const uint32_t* terms, const int e[3], uint32_t M, std::vector<uint32_t>& d);

// Checks a word buffer against the layout of `spec` (pointers inside the
// buffer, masks, DF distances); fills the per-level word and node counts.
int validate_canonical(const Spec& spec, const uint32_t* words, uint64_t n, BuildResult* stats);

// Device image (pack.cpp): the canonical structures relocated so that
// two-word structures start at even words, pointers rewritten; *packed is
// set when SVDAG pointers also carry masks (images below 2^24 words with an
// SVDAG level).  False when the buffer is not a well-formed volume of the
// spec (then the canonical words are uploaded as they are).
// stage_end (optional, kStageLevels + 1 words): stage_end[k] = the image's
// words before the first structure read at node level k or deeper (the top
// k node levels are the prefix [0, stage_end[k])).
constexpr int kStageLevels = 8;
bool make_device_image(const Spec& spec, const std::vector<uint32_t>& canonical, std::vector<uint32_t>& out,
                       bool* packed, uint32_t* stage_end = nullptr);

// Decodes the cube (side 2^log2s at x0,y0,z0) from a canonical buffer.
int decode_cube(const Spec& spec, const uint32_t* words, uint64_t nwords, int64_t x0, int64_t y0, int64_t z0,
                int log2s, uint32_t* out);

// ---------------------------------------------------------------------------
// Device side
// ---------------------------------------------------------------------------
struct CameraParams {
    float eye[3];
    float f[3], r[3], u[3];
    float tha, th;  // tan(vfov/2) * W/H, tan(vfov/2)
    uint32_t W, H;
};

struct KernelSet;  // kernels for one format (trace.cuh)

// Device buffers and streams of the *_host calls (chunked copy/trace pipeline).
// kDepth chunks in flight on kDepth streams: the upload of one chunk, the
// kernel of another and the download of a third overlap (PCIe moves data both
// ways at once).
struct Staging {
    static constexpr uint64_t kChunk = 1u << 18;  // rays per chunk
    static constexpr int kDepth = 4;
    void* d_rays[kDepth] = {};
    void* d_hits[kDepth] = {};
    void* streams[kDepth] = {};
    void* ready = nullptr;
};

constexpr int kDefaultRefill = 8;  // persistent kernel: idle lanes before a warp refills
constexpr int kDefaultBurst = 4;   // persistent kernel: iterations between refill checks
// Batched calls without vx_autotune_batch: the same options for every group.
// Over a grid of block {128, 256} x refill {2..16} x burst {8, 16, 32} on the
// 2048^3 batched workload, blocks of 256 with refill 4 and burst 16 were
// fastest (2075 Mrays/s; refill 8 / burst 4: 1987).
constexpr int kBatchRefill = 4;
constexpr int kBatchBurst = 16;
constexpr int kQueueRing = 256;      // queue counters per volume for launches issued directly
constexpr int kQueueCaptured = 3840;  // further counters, each given to one captured launch for good

struct Volume {
    Spec spec;
    BuildResult built;
    vx_stats stats{};
    int device = -1;
    uint32_t* d_pool = nullptr;
    uint64_t pool_words = 0;
    int packed = 0;   // device image in the packed layout (pack.cpp)
    int aligned = 0;  // device image with two-word structures at even words (pack.cpp)
    uint32_t stage_end[kStageLevels + 1] = {};  // prefix of the image holding the top k node levels
    bool unvalidated = false;  // loaded without validation: only the checked (counted) trace may read it
    const KernelSet* kernels = nullptr;
    std::mutex staging_mu;
    Staging staging;
    std::mutex tune_mu;
    bool tuned = false;
    vx_trace_opts tuned_opts{};             // chosen by vx_autotune, used for VX_MODE_AUTO
    bool batch_tuned = false;
    vx_trace_opts tuned_batch{};            // chosen by vx_autotune_batch for this volume's batched group
    unsigned long long* d_queue = nullptr;  // kQueueRing + kQueueCaptured counters
    mutable std::atomic<uint32_t> queue_slot{0};
    mutable std::atomic<uint32_t> captured_slot{0};
    // The ray-queue counter of one persistent launch on `stream`.  A launch
    // issued directly takes the next counter of a ring of kQueueRing, so up
    // to kQueueRing of them may be in flight at once per volume.  A launch
    // being captured into a CUDA graph keeps its counter for every replay,
    // so it gets one of the kQueueCaptured counters that no other launch
    // ever uses; nullptr once they are used up (or without a device image).
    unsigned long long* queue_counter(void* stream) const;
};

const KernelSet* kernels_for(const Spec& sp);
uint32_t stage_words(const Volume& v, int k);  // image words staged for smem_top = k (launch.cu)
bool kernel_set_specialized(const KernelSet* k);

// Kernel registry: compile-time-composed kernels for known signatures, and
// the run-time-described kernels for any other signature.
const KernelSet* find_kernels(const std::string& canonical_spec);
const KernelSet* generic_kernels();
std::vector<const KernelSet*> registered_kernel_sets();  // compile-time-composed sets, in registration order
const char* kernel_set_spec(const KernelSet* k);

int launch_trace(const Volume& v, const vx_ray* rays, uint64_t n, void* hits, int layout, const vx_trace_opts* o,
                 void* stream);
int launch_trace_count(const Volume& v, const vx_ray* rays, uint64_t n, void* hits, int layout,
                       const vx_trace_opts* o, void* stream, unsigned long long* counters, uint32_t* sectors);
int launch_render(const Volume& v, const CameraParams& cp, uint64_t i0, uint64_t n, void* hits, int layout,
                  const vx_trace_opts* o, void* stream);
// count views of one volume; view k renders pixels [i0[k], i0[k] + n[k]) of
// camera k into hits[k] (plain mode: up to 16 views per launch)
int launch_render_views(const Volume& v, const CameraParams* cps, const uint64_t* i0, const uint64_t* n,
                        void* const* hits, int count, int layout, const vx_trace_opts* o, void* stream);
int launch_raygen(const CameraParams& cp, vx_ray* rays, void* stream);
int launch_ao(const vx_ray* rays, const void* hits, uint64_t n, uint64_t seed, int spp, float eps, float tmax,
              vx_ray* out, void* stream);
struct BatchItemIn {
    const Volume* v;
    const vx_ray* rays;
    uint64_t n;
    void* hits;
};
// events: optional, n_events caller-created events recorded around group k's
// kernel (2k before, 2k + 1 after) on its stream; *groups receives the count.
int launch_batch(const std::vector<BatchItemIn>& items, int layout, const vx_trace_opts* o, void* stream,
                 void** events = nullptr, uint32_t n_events = 0, uint32_t* groups = nullptr);
// The same sets with rays and hits in host memory, streamed through the device
// in waves; returns when every hit is in host memory.
int launch_batch_host(const std::vector<BatchItemIn>& items, int layout, const vx_trace_opts* o, void* stream);
// Coherence sort (sort.cu): rays copied in key order into scratch, space for
// their hits in that order, and each ray's position.
struct SortedRays {
    const vx_ray* rays = nullptr;
    void* hits = nullptr;
    const uint32_t* pos = nullptr;
};
uint64_t sort_scratch_bytes(const int ldim[3], int g, uint64_t n, uint32_t hit_bytes, uint32_t* nbins_out);
int sort_rays(const int ldim[3], int g, const vx_ray* rays, uint64_t n, uint32_t hit_bytes, void* scratch,
              SortedRays* out, struct CUstream_st* st);
int unsort_hits(const SortedRays& s, uint64_t n, void* hits, int layout, struct CUstream_st* st);
int trace_noalloc(const Volume& v, const vx_ray* rays, uint64_t n, void* hits, int layout, void* stream);
int camera_params(const vx_camera* cam, CameraParams* out);

}  // namespace vx
