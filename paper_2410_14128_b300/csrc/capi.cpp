// capi.cpp -- the extern "C" entry points declared in include/vx.h.
#include <cuda_runtime.h>
#include <string.h>

#include <algorithm>
#include <chrono>
#include <memory>

#include "vx_internal.hpp"

using namespace vx;

struct vx_volume_s {
    Volume v;
};

namespace {

double now_ms() {
    using namespace std::chrono;
    return duration<double, std::milli>(steady_clock::now().time_since_epoch()).count();
}

int cuda_fail(cudaError_t e, const char* what) {
    return fail(e == cudaErrorMemoryAllocation ? VX_ENOMEM : VX_ECUDA, "%s: %s", what, cudaGetErrorString(e));
}

// Makes the volume's device current for the scope of a call.
class DeviceScope {
  public:
    explicit DeviceScope(int dev) {
        cudaGetDevice(&prev_);
        if (dev >= 0 && dev != prev_) {
            err_ = cudaSetDevice(dev);
            changed_ = err_ == cudaSuccess;
        }
    }
    ~DeviceScope() {
        if (changed_) cudaSetDevice(prev_);
    }
    cudaError_t error() const { return err_; }

  private:
    int prev_ = 0;
    bool changed_ = false;
    cudaError_t err_ = cudaSuccess;
};

bool aligned(const void* p, size_t a) { return ((uintptr_t)p % a) == 0; }

// checked: the caller is the instrumented trace, whose reads are checked
// against the image size, so it may read a volume loaded without validation.
int check_trace_args(vx_volume v, const void* rays, uint64_t n, const void* hits, int32_t layout,
                     bool checked = false) {
    if (!v) return fail(VX_EINVAL, "volume is NULL");
    if (!v->v.d_pool) return fail(VX_EINVAL, "volume has no device image (built with no_upload)");
    if (v->v.unvalidated && !checked)
        return fail(VX_EINVAL, "volume was loaded without validation: only vx_trace_counted may trace it");
    if (layout != VX_HIT_FULL && layout != VX_HIT_COMPACT) return fail(VX_EINVAL, "bad hit layout %d", layout);
    if (layout == VX_HIT_COMPACT && v->v.spec.ldim[0] + v->v.spec.ldim[1] + v->v.spec.ldim[2] >= 32)
        return fail(VX_EINVAL, "compact hits need fewer than 2^32 voxels");
    if (n == 0) return VX_OK;
    return VX_OK;
}

int check_opts(const vx_trace_opts* o) {
    if (!o) return VX_OK;
    if (o->block != 0 && (o->block < 32 || o->block > 256 || (o->block & 31)))
        return fail(VX_EINVAL, "block must be 0 or a multiple of 32 in [32, 256], got %d", o->block);
    if (o->mode < VX_MODE_AUTO || o->mode > VX_MODE_PERSISTENT) return fail(VX_EINVAL, "bad mode %d", o->mode);
    if (o->refill < 0 || o->refill > 32) return fail(VX_EINVAL, "refill must be in [0, 32], got %d", o->refill);
    if (o->burst < 0 || o->burst > 1024) return fail(VX_EINVAL, "burst must be in [0, 1024], got %d", o->burst);
    if (o->sort_cell_log2 < 0 || o->sort_cell_log2 > 15)
        return fail(VX_EINVAL, "sort_cell_log2 must be in [0, 15], got %d", o->sort_cell_log2);
    if (o->blocks_per_sm < 0 || o->blocks_per_sm > 32)
        return fail(VX_EINVAL, "blocks_per_sm must be in [0, 32], got %d", o->blocks_per_sm);
    if (o->restart != 0 && o->restart != 1) return fail(VX_EINVAL, "restart must be 0 or 1, got %d", o->restart);
    if (o->smem_top < 0 || o->smem_top > kStageLevels)
        return fail(VX_EINVAL, "smem_top must be in [0, %d], got %d", kStageLevels, o->smem_top);
    if (o->short_stack != 0 && o->short_stack != 1 && o->short_stack != 2 && o->short_stack != 4 &&
        o->short_stack != 8)
        return fail(VX_EINVAL, "short_stack must be 0, 1, 2, 4 or 8, got %d", o->short_stack);
    if (o->short_stack && o->restart) return fail(VX_EINVAL, "short_stack and restart exclude each other");
    return VX_OK;
}

int check_ptrs(const void* rays, const void* hits, int32_t layout) {
    if (rays && !aligned(rays, 16)) return fail(VX_EINVAL, "rays must be 16-byte aligned");
    if (!hits) return fail(VX_EINVAL, "hits is NULL");
    if (!aligned(hits, layout == VX_HIT_FULL ? 16 : 8)) return fail(VX_EINVAL, "hits misaligned for the layout");
    return VX_OK;
}

size_t hit_bytes(int layout) { return layout == VX_HIT_FULL ? sizeof(vx_hit) : sizeof(vx_hit_compact); }

int ensure_staging(Volume& V) {
    Staging& S = V.staging;
    if (S.ready) return VX_OK;
    for (int i = 0; i < Staging::kDepth; i++) {
        cudaError_t e = cudaMalloc(&S.d_rays[i], Staging::kChunk * sizeof(vx_ray));
        if (e) return cuda_fail(e, "cudaMalloc (staging rays)");
        e = cudaMalloc(&S.d_hits[i], Staging::kChunk * sizeof(vx_hit));
        if (e) return cuda_fail(e, "cudaMalloc (staging hits)");
        cudaStream_t st;
        e = cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking);
        if (e) return cuda_fail(e, "cudaStreamCreate");
        S.streams[i] = st;
    }
    cudaEvent_t ev;
    cudaError_t e = cudaEventCreateWithFlags(&ev, cudaEventDisableTiming);
    if (e) return cuda_fail(e, "cudaEventCreate");
    S.ready = ev;
    return VX_OK;
}

void free_staging(Staging& S) {
    for (int i = 0; i < Staging::kDepth; i++) {
        if (S.d_rays[i]) cudaFree(S.d_rays[i]);
        if (S.d_hits[i]) cudaFree(S.d_hits[i]);
        if (S.streams[i]) cudaStreamDestroy((cudaStream_t)S.streams[i]);
        S.d_rays[i] = S.d_hits[i] = S.streams[i] = nullptr;
    }
    if (S.ready) cudaEventDestroy((cudaEvent_t)S.ready);
    S.ready = nullptr;
}

// Runs `work(i0, n, d_rays, d_hits, stream)` over chunks of the input on
// Staging::kDepth streams in turn, so copies in both directions overlap the
// kernels of other chunks.
template <class Work>
int pipeline(Volume& V, uint64_t n, void* stream, Work work) {
    // the call waits for its copies, which a stream capture cannot hold
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    cudaError_t ce = cudaStreamIsCapturing((cudaStream_t)stream, &cs);
    if (ce) return cuda_fail(ce, "cudaStreamIsCapturing");
    if (cs != cudaStreamCaptureStatusNone)
        return fail(VX_EUNSUPPORTED, "tracing from host memory waits for its copies: not on a capturing stream");
    std::lock_guard<std::mutex> lock(V.staging_mu);
    int rc = ensure_staging(V);
    if (rc) return rc;
    Staging& S = V.staging;
    cudaEvent_t ready = (cudaEvent_t)S.ready;
    cudaError_t e = cudaEventRecord(ready, (cudaStream_t)stream);
    if (e) return cuda_fail(e, "cudaEventRecord");
    for (int i = 0; i < Staging::kDepth; i++) {
        e = cudaStreamWaitEvent((cudaStream_t)S.streams[i], ready, 0);
        if (e) return cuda_fail(e, "cudaStreamWaitEvent");
    }
    uint64_t k = 0;
    for (uint64_t i0 = 0; i0 < n; i0 += Staging::kChunk, k++) {
        const uint64_t m = (n - i0) < Staging::kChunk ? (n - i0) : Staging::kChunk;
        const int b = (int)(k % Staging::kDepth);
        rc = work(i0, m, S.d_rays[b], S.d_hits[b], (cudaStream_t)S.streams[b]);
        if (rc) break;
    }
    for (int i = 0; i < Staging::kDepth; i++) {
        e = cudaStreamSynchronize((cudaStream_t)S.streams[i]);
        if (e && !rc) rc = cuda_fail(e, "trace pipeline");
    }
    return rc;
}

}  // namespace

namespace {
// Device image (packed when allowed and possible) and queue counters.
int upload(Volume& V, const vx_build_opts& o, bool allow_packed) {
    int dev = o.device;
    if (dev < 0) {
        cudaError_t e = cudaGetDevice(&dev);
        if (e) return cuda_fail(e, "cudaGetDevice");
    }
    DeviceScope ds(dev);
    if (ds.error()) return cuda_fail(ds.error(), "cudaSetDevice");
    V.device = dev;
    std::vector<uint32_t> image;
    bool packed = false;
    const bool relocated = allow_packed && make_device_image(V.spec, V.built.words, image, &packed, V.stage_end);
    V.packed = relocated && packed ? 1 : 0;
    V.aligned = relocated ? 1 : 0;
    const std::vector<uint32_t>& src = relocated ? image : V.built.words;
    const uint64_t bytes = src.size() * sizeof(uint32_t);
    cudaError_t e = cudaMalloc((void**)&V.d_pool, bytes);
    if (e) return cuda_fail(e, "cudaMalloc (device image)");
    e = cudaMemcpy(V.d_pool, src.data(), bytes, cudaMemcpyHostToDevice);
    if (e) { cudaFree(V.d_pool); V.d_pool = nullptr; return cuda_fail(e, "cudaMemcpy (device image)"); }
    V.pool_words = src.size();
    e = cudaMalloc((void**)&V.d_queue, (kQueueRing + kQueueCaptured) * sizeof(unsigned long long));
    if (e) { cudaFree(V.d_pool); V.d_pool = nullptr; return cuda_fail(e, "cudaMalloc (queue counters)"); }
    V.stats.device_bytes = bytes;
    V.stats.packed = V.packed;
    V.stats.aligned = V.aligned;
    return VX_OK;
}
}  // namespace

extern "C" int vx_build(const char* spec, const vx_grid* grid, const vx_build_opts* opts, vx_volume* out) {
    clear_error();
    if (!out) return fail(VX_EINVAL, "out is NULL");
    *out = nullptr;
    Spec sp;
    int rc = parse_spec(spec, &sp);
    if (rc) return rc;
    if (!grid) return fail(VX_EINVAL, "grid is NULL");
    if ((grid->dense != nullptr) + (grid->fill_brick != nullptr) + (grid->dense_pal != nullptr) != 1)
        return fail(VX_EINVAL, "set exactly one of grid->dense, grid->dense_pal and grid->fill_brick");
    if (grid->dense_pal && (!grid->palette || grid->palette[0] != 0))
        return fail(VX_EINVAL, "grid->dense_pal needs a palette whose entry 0 is 0 (empty)");
    for (int i = 0; i < 3; i++)
        if ((int)grid->log2_dim[i] != sp.ldim[i])
            return fail(VX_EINVAL, "spec '%s' describes a 2^%d x 2^%d x 2^%d grid, the grid is 2^%u x 2^%u x 2^%u",
                        spec, sp.ldim[0], sp.ldim[1], sp.ldim[2], grid->log2_dim[0], grid->log2_dim[1],
                        grid->log2_dim[2]);
    vx_build_opts o{VX_DEDUP_WHOLE_LEVEL, -1, 0, 0, 0, 0, {0, 0}};
    if (opts) o = *opts;
    if (o.dedup_scope != VX_DEDUP_WHOLE_LEVEL && o.dedup_scope != VX_DEDUP_PER_SUBVOLUME)
        return fail(VX_EINVAL, "bad dedup_scope %d", o.dedup_scope);

    std::unique_ptr<vx_volume_s> h(new vx_volume_s);
    Volume& V = h->v;
    V.spec = sp;
    const double t0 = now_ms();
    std::unique_ptr<VoxelSource> src(grid->dense       ? make_dense_source(grid->dense, sp.ldim)
                                     : grid->dense_pal ? make_palette_source(grid->dense_pal, grid->palette, sp.ldim)
                                                       : make_brick_source(grid));
    rc = build_canonical(sp, *src, o.dedup_scope, &V.built, o.threads);
    if (rc) return rc;
    const double t1 = now_ms();

    vx_stats& st = V.stats;
    memset(&st, 0, sizeof st);
    st.n_levels = (uint32_t)sp.lv.size();
    st.n_node_levels = sp.fmt.J;
    for (int i = 0; i < 3; i++) st.log2_dim[i] = (uint32_t)sp.ldim[i];
    st.canonical_words = V.built.words.size();
    st.occupied_voxels = V.built.occupied;
    for (int k = 0; k < VX_MAX_LEVELS; k++) {
        st.level_words[k] = V.built.level_words[k];
        st.level_nodes[k] = V.built.level_nodes[k];
    }
    st.build_ms = t1 - t0;
    V.kernels = o.generic_kernel ? generic_kernels() : kernels_for(sp);
    st.specialized = kernel_set_specialized(V.kernels) ? 1 : 0;

    if (!o.no_upload) {
        rc = upload(V, o, !o.canonical_device);
        if (rc) return rc;
        st.upload_ms = now_ms() - t1;
    }
    *out = h.release();
    return VX_OK;
}

extern "C" int vx_load(const char* spec, const uint32_t* words, uint64_t n_words, const vx_build_opts* opts,
                       int32_t validate, vx_volume* out) {
    clear_error();
    if (!out) return fail(VX_EINVAL, "out is NULL");
    *out = nullptr;
    if (!words || n_words == 0) return fail(VX_EINVAL, "words is empty");
    if (n_words > 0xFFFFFFFFull) return fail(VX_ETOOBIG, "buffer exceeds 2^32 words (16 GiB, Sec. 3.3)");
    Spec sp;
    int rc = parse_spec(spec, &sp);
    if (rc) return rc;
    vx_build_opts o{VX_DEDUP_WHOLE_LEVEL, -1, 0, 0, 0, 0, {0, 0}};
    if (opts) o = *opts;
    std::unique_ptr<vx_volume_s> h(new vx_volume_s);
    Volume& V = h->v;
    V.spec = sp;
    const double t0 = now_ms();
    V.built.words.assign(words, words + n_words);
    if (validate) {
        rc = validate_canonical(sp, V.built.words.data(), n_words, &V.built);
        if (rc) return rc;
    } else {
        V.unvalidated = true;
    }
    vx_stats& st = V.stats;
    memset(&st, 0, sizeof st);
    st.n_levels = (uint32_t)sp.lv.size();
    st.n_node_levels = sp.fmt.J;
    for (int i = 0; i < 3; i++) st.log2_dim[i] = (uint32_t)sp.ldim[i];
    st.canonical_words = n_words;
    for (int k = 0; k < VX_MAX_LEVELS; k++) {
        st.level_words[k] = V.built.level_words[k];
        st.level_nodes[k] = V.built.level_nodes[k];
    }
    st.build_ms = now_ms() - t0;
    V.kernels = o.generic_kernel ? generic_kernels() : kernels_for(sp);
    st.specialized = kernel_set_specialized(V.kernels) ? 1 : 0;
    if (!o.no_upload) {
        const double t1 = now_ms();
        // an unvalidated buffer is uploaded as it is: the packer trusts the layout
        rc = upload(V, o, validate && !o.canonical_device);
        if (rc) return rc;
        st.upload_ms = now_ms() - t1;
    }
    *out = h.release();
    return VX_OK;
}

extern "C" int vx_formats(const char** specs, uint32_t capacity, uint32_t* count) {
    clear_error();
    if (!count) return fail(VX_EINVAL, "count is NULL");
    const std::vector<const KernelSet*> all = registered_kernel_sets();
    *count = (uint32_t)all.size();
    if (specs)
        for (uint32_t i = 0; i < capacity && i < all.size(); i++) specs[i] = kernel_set_spec(all[i]);
    return VX_OK;
}

extern "C" int vx_free(vx_volume v) {
    clear_error();
    if (!v) return VX_OK;
    {
        DeviceScope ds(v->v.device);
        if (v->v.d_pool) {
            cudaDeviceSynchronize();
            cudaFree(v->v.d_pool);
        }
        if (v->v.d_queue) cudaFree(v->v.d_queue);
        free_staging(v->v.staging);
    }
    delete v;
    return VX_OK;
}

extern "C" int vx_stats_get(vx_volume v, vx_stats* out) {
    clear_error();
    if (!v || !out) return fail(VX_EINVAL, "NULL argument");
    *out = v->v.stats;
    std::lock_guard<std::mutex> lock(v->v.tune_mu);
    out->tuned = v->v.tuned ? 1 : 0;
    out->tuned_opts = v->v.tuned ? v->v.tuned_opts : vx_trace_opts{};
    return VX_OK;
}

extern "C" int vx_canonical(vx_volume v, const uint32_t** words, uint64_t* n_words) {
    clear_error();
    if (!v || !words || !n_words) return fail(VX_EINVAL, "NULL argument");
    *words = v->v.built.words.data();
    *n_words = v->v.built.words.size();
    return VX_OK;
}

extern "C" int vx_decode_brick(vx_volume v, uint32_t x0, uint32_t y0, uint32_t z0, uint32_t log2_size, uint32_t* out) {
    clear_error();
    if (!v || !out) return fail(VX_EINVAL, "NULL argument");
    const Spec& sp = v->v.spec;
    const uint32_t c[3] = {x0, y0, z0};
    for (int i = 0; i < 3; i++) {
        if ((int)log2_size > sp.ldim[i]) return fail(VX_EINVAL, "cube larger than the grid");
        if (c[i] & ((1u << log2_size) - 1u)) return fail(VX_EINVAL, "cube corner not a multiple of its side");
        if ((uint64_t)c[i] + (1ull << log2_size) > (1ull << sp.ldim[i])) return fail(VX_EINVAL, "cube outside the grid");
    }
    memset(out, 0, sizeof(uint32_t) << (3 * log2_size));
    return decode_cube(sp, v->v.built.words.data(), v->v.built.words.size(), x0, y0, z0, (int)log2_size, out);
}

extern "C" int vx_trace(vx_volume v, const vx_ray* rays, uint64_t n, void* hits, int32_t hit_layout,
                        const vx_trace_opts* opts, void* stream) {
    clear_error();
    int rc = check_trace_args(v, rays, n, hits, hit_layout);
    if (!rc) rc = check_opts(opts);
    if (rc || n == 0) return rc;
    if ((rc = check_ptrs(rays, hits, hit_layout))) return rc;
    if (!rays) return fail(VX_EINVAL, "rays is NULL");
    DeviceScope ds(v->v.device);
    if (ds.error()) return cuda_fail(ds.error(), "cudaSetDevice");
    return launch_trace(v->v, rays, n, hits, hit_layout, opts, stream);
}

extern "C" int vx_trace_counted(vx_volume v, const vx_ray* rays, uint64_t n, void* hits, int32_t hit_layout,
                                const vx_trace_opts* opts, void* stream, unsigned long long* counters,
                                uint32_t* sectors) {
    clear_error();
    int rc = check_trace_args(v, rays, n, hits, hit_layout, true);
    if (!rc) rc = check_opts(opts);
    if (rc || n == 0) return rc;
    if ((rc = check_ptrs(rays, hits, hit_layout))) return rc;
    if (!rays) return fail(VX_EINVAL, "rays is NULL");
    if (!counters || !aligned(counters, 8)) return fail(VX_EINVAL, "counters must be an 8-byte aligned device array");
    if (sectors && !aligned(sectors, 4)) return fail(VX_EINVAL, "sectors must be a 4-byte aligned device array");
    DeviceScope ds(v->v.device);
    if (ds.error()) return cuda_fail(ds.error(), "cudaSetDevice");
    return launch_trace_count(v->v, rays, n, hits, hit_layout, opts, stream, counters, sectors);
}

extern "C" int vx_trace_batch(const vx_batch_item* items, uint32_t count, int32_t hit_layout,
                              const vx_trace_opts* opts, void* stream) {
    return vx_trace_batch_timed(items, count, hit_layout, opts, stream, nullptr, 0, nullptr);
}

extern "C" int vx_trace_batch_timed(const vx_batch_item* items, uint32_t count, int32_t hit_layout,
                                    const vx_trace_opts* opts, void* stream, void** events, uint32_t n_events,
                                    uint32_t* groups) {
    clear_error();
    if (groups) *groups = 0;
    if (n_events > 0 && !events) return fail(VX_EINVAL, "events is NULL");
    if (count == 0) return VX_OK;
    if (!items) return fail(VX_EINVAL, "items is NULL");
    if (count > 65536) return fail(VX_EINVAL, "at most 65536 items per batch");
    int rc = check_opts(opts);
    if (rc) return rc;
    if (opts && opts->sort_cell_log2 != 0) return fail(VX_EUNSUPPORTED, "batched tracing does not sort rays");
    int dev = -1;
    std::vector<BatchItemIn> in;
    in.reserve(count);
    for (uint32_t i = 0; i < count; i++) {
        const vx_batch_item& it = items[i];
        rc = check_trace_args(it.volume, it.rays, it.n, it.hits, hit_layout);
        if (rc) return fail(rc, "item %u: %s", i, vx_last_error());
        if (it.n == 0) continue;
        if ((rc = check_ptrs(it.rays, it.hits, hit_layout))) return fail(rc, "item %u: %s", i, vx_last_error());
        if (!it.rays) return fail(VX_EINVAL, "item %u: rays is NULL", i);
        if (dev < 0) dev = it.volume->v.device;
        else if (it.volume->v.device != dev) return fail(VX_EINVAL, "item %u: all volumes must be on one device", i);
        in.push_back(BatchItemIn{&it.volume->v, it.rays, it.n, it.hits});
    }
    if (in.empty()) return VX_OK;
    DeviceScope ds(dev);
    if (ds.error()) return cuda_fail(ds.error(), "cudaSetDevice");
    return launch_batch(in, hit_layout, opts, stream, events, n_events, groups);
}

extern "C" int vx_trace_batch_host(const vx_batch_item* items, uint32_t count, int32_t hit_layout,
                                   const vx_trace_opts* opts, void* stream) {
    clear_error();
    if (count == 0) return VX_OK;
    if (!items) return fail(VX_EINVAL, "items is NULL");
    if (count > 65536) return fail(VX_EINVAL, "at most 65536 items per batch");
    int rc = check_opts(opts);
    if (rc) return rc;
    if (opts && opts->sort_cell_log2 != 0) return fail(VX_EUNSUPPORTED, "batched tracing does not sort rays");
    int dev = -1;
    std::vector<BatchItemIn> in;
    in.reserve(count);
    for (uint32_t i = 0; i < count; i++) {
        const vx_batch_item& it = items[i];
        rc = check_trace_args(it.volume, it.rays, it.n, it.hits, hit_layout);
        if (rc) return fail(rc, "item %u: %s", i, vx_last_error());
        if (it.n == 0) continue;
        if ((rc = check_ptrs(it.rays, it.hits, hit_layout))) return fail(rc, "item %u: %s", i, vx_last_error());
        if (!it.rays) return fail(VX_EINVAL, "item %u: rays is NULL", i);
        if (dev < 0) dev = it.volume->v.device;
        else if (it.volume->v.device != dev) return fail(VX_EINVAL, "item %u: all volumes must be on one device", i);
        in.push_back(BatchItemIn{&it.volume->v, it.rays, it.n, it.hits});
    }
    if (in.empty()) return VX_OK;
    DeviceScope ds(dev);
    if (ds.error()) return cuda_fail(ds.error(), "cudaSetDevice");
    return launch_batch_host(in, hit_layout, opts, stream);
}

// ---------------------------------------------------------------------------
// Autotuner: coordinate descent over the trace options, each candidate timed
// with CUDA events on the sample (best of 3 runs after one warm-up run).
// ---------------------------------------------------------------------------
namespace {

int time_opts(Volume& V, const vx_ray* rays, uint64_t n, void* hits, const vx_trace_opts& o, cudaStream_t st,
              cudaEvent_t a, cudaEvent_t b, float* ms) {
    int rc = launch_trace(V, rays, n, hits, VX_HIT_FULL, &o, st);
    if (rc) return rc;
    float best = 1e30f;
    for (int r = 0; r < 3; r++) {
        cudaEventRecord(a, st);
        rc = launch_trace(V, rays, n, hits, VX_HIT_FULL, &o, st);
        if (rc) return rc;
        cudaEventRecord(b, st);
        cudaError_t e = cudaEventSynchronize(b);
        if (e) return cuda_fail(e, "autotune");
        float t = 0.0f;
        cudaEventElapsedTime(&t, a, b);
        if (t < best) best = t;
    }
    *ms = best;
    return VX_OK;
}

}  // namespace

extern "C" int vx_autotune(vx_volume v, const vx_ray* rays, uint64_t n, void* stream, vx_trace_opts* best_out,
                           double* best_ms) {
    clear_error();
    int rc = check_trace_args(v, rays, n, nullptr, VX_HIT_FULL);
    if (rc) return rc;
    if (n == 0 || !rays) return fail(VX_EINVAL, "autotune needs a non-empty sample of rays");
    if (!aligned(rays, 16)) return fail(VX_EINVAL, "rays must be 16-byte aligned");
    DeviceScope ds(v->v.device);
    if (ds.error()) return cuda_fail(ds.error(), "cudaSetDevice");
    Volume& V = v->v;
    cudaStream_t st = (cudaStream_t)stream;
    void* hits = nullptr;
    cudaError_t e = cudaMalloc(&hits, n * sizeof(vx_hit));
    if (e) return cuda_fail(e, "cudaMalloc (autotune hits)");
    cudaEvent_t a, b;
    cudaEventCreate(&a);
    cudaEventCreate(&b);
    vx_trace_opts cur{};
    cur.mode = VX_MODE_PERSISTENT;
    cur.block = 256;
    cur.refill = kDefaultRefill;
    cur.burst = kDefaultBurst;
    float cur_ms = 0.0f;
    rc = time_opts(V, rays, n, hits, cur, st, a, b, &cur_ms);
    auto consider = [&](vx_trace_opts cand) {
        if (rc) return;
        float ms = 0.0f;
        rc = time_opts(V, rays, n, hits, cand, st, a, b, &ms);
        // a candidate replaces the current options only when it is more than
        // 1% faster: best-of-3 timings of a sub-millisecond sample differ by
        // about that much between repeats, and a near-tie keeps the options
        // reached first (fewer kernels: no sort, no restart)
        if (!rc && ms < cur_ms * 0.99f) { cur = cand; cur_ms = ms; }
    };
    // restarting traversal differs from the stack only below an octree
    // level's root, i.e. for SVO / SVDAG levels of depth 2 or more
    bool deep_octree = false;
    for (const Level& L : V.spec.lv) deep_octree |= (L.kind == K_SVO || L.kind == K_DAG) && L.e[0] >= 2;
    if (deep_octree) { vx_trace_opts c = cur; c.restart = 1; consider(c); }
    // a short stack between the two: the ring only matters below an octree
    // level's root, for octree levels deeper than the ring
    int deepest = 0;
    for (const Level& L : V.spec.lv)
        if (L.kind == K_SVO || L.kind == K_DAG) deepest = std::max(deepest, L.e[0]);
    for (int d : {1, 2, 4}) {
        if (d + 1 >= deepest || cur.restart) break;
        vx_trace_opts c = cur;
        c.short_stack = d;
        consider(c);
    }
    // staging depth: the top k node levels in shared memory, for each k whose
    // image prefix fits and differs from the previous one
    if (!cur.restart && !cur.short_stack) {
        uint32_t last = 0;
        for (int k = 1; k <= kStageLevels; k++) {
            const uint32_t w = stage_words(V, k);
            if (w == 0 || w == last) continue;
            last = w;
            vx_trace_opts c = cur;
            c.smem_top = k;
            consider(c);
        }
    }
    // sort granularities; the key keeps at most 5 bits per axis, so at large
    // grids several g give the same key cells (tried once)
    const int maxg = std::min(V.spec.ldim[0], std::min(V.spec.ldim[1], V.spec.ldim[2]));
    int last_shift = -1;
    for (int g : {2, 3, 4, 5, 6, 7}) {
        if (g > maxg) break;
        int shift = 0;
        for (int i = 0; i < 3; i++) {
            const int b = std::min(std::max(V.spec.ldim[i] - g, 0), 5);
            shift = shift * 16 + (V.spec.ldim[i] - b);
        }
        if (shift == last_shift) continue;
        last_shift = shift;
        vx_trace_opts c = cur; c.sort_cell_log2 = g; consider(c);
    }
    // two rounds of coordinate descent over the persistent-kernel knobs (a
    // knob's best value can move once the others have)
    for (int round = 0; round < 2; round++) {
        for (int r : {1, 2, 4, 8, 16, 24, 32}) { vx_trace_opts c = cur; c.refill = r; consider(c); }
        for (int bu : {1, 2, 4, 8, 16, 32, 64}) { vx_trace_opts c = cur; c.burst = bu; consider(c); }
        for (int bl : {64, 128, 256}) { vx_trace_opts c = cur; c.block = bl; consider(c); }
    }
    // the one-thread-per-ray kernel (sorting and restarting carry over;
    // shared-memory staging is a persistent-kernel option)
    {
        const vx_trace_opts p = cur;
        for (int bl : {64, 128, 256}) {
            vx_trace_opts c = p;
            c.mode = VX_MODE_PLAIN;
            c.smem_top = 0;
            c.block = bl;
            consider(c);
        }
    }
    cudaEventDestroy(a);
    cudaEventDestroy(b);
    cudaFree(hits);
    if (rc) return rc;
    {
        std::lock_guard<std::mutex> lock(V.tune_mu);
        V.tuned_opts = cur;
        V.tuned = true;
    }
    if (best_out) *best_out = cur;
    if (best_ms) *best_ms = cur_ms;
    return VX_OK;
}

// Batched-launch autotuner.  The objective is the whole batched call: the
// groups' kernels run concurrently and share the SMs, so a group's options
// are judged by the time of the call, not of the group alone.  Coordinate
// descent over the batched kernel's refill threshold, burst and block size,
// first for all volumes at once (two rounds), then per volume with the
// others fixed (one round); each candidate timed as the whole call (best of
// three after one warm-up call), replacing the current options only when
// more than 1% faster.
extern "C" int vx_autotune_batch(const vx_batch_item* items, uint32_t count, int32_t hit_layout, void* stream,
                                 vx_trace_opts* chosen) {
    clear_error();
    if (count == 0) return VX_OK;
    if (!items) return fail(VX_EINVAL, "items is NULL");
    if (count > 65536) return fail(VX_EINVAL, "at most 65536 items per batch");
    int dev = -1;
    std::vector<BatchItemIn> in;
    std::vector<Volume*> vols;  // distinct volumes, in order of first appearance
    for (uint32_t i = 0; i < count; i++) {
        const vx_batch_item& it = items[i];
        int rc = check_trace_args(it.volume, it.rays, it.n, it.hits, hit_layout);
        if (rc) return fail(rc, "item %u: %s", i, vx_last_error());
        if (it.n == 0) continue;
        if ((rc = check_ptrs(it.rays, it.hits, hit_layout))) return fail(rc, "item %u: %s", i, vx_last_error());
        if (!it.rays) return fail(VX_EINVAL, "item %u: rays is NULL", i);
        if (dev < 0) dev = it.volume->v.device;
        else if (it.volume->v.device != dev) return fail(VX_EINVAL, "item %u: all volumes must be on one device", i);
        in.push_back(BatchItemIn{&it.volume->v, it.rays, it.n, it.hits});
        if (std::find(vols.begin(), vols.end(), &it.volume->v) == vols.end()) vols.push_back(&it.volume->v);
    }
    if (in.empty()) return VX_OK;
    DeviceScope ds(dev);
    if (ds.error()) return cuda_fail(ds.error(), "cudaSetDevice");
    cudaStream_t st = (cudaStream_t)stream;
    cudaEvent_t a = nullptr, b = nullptr;
    cudaError_t ce = cudaEventCreate(&a);
    if (!ce) ce = cudaEventCreate(&b);
    if (ce) {
        if (a) cudaEventDestroy(a);
        return cuda_fail(ce, "cudaEventCreate");
    }
    // the options each volume's group uses now; the candidate assignment is
    // installed as the volumes' batched options while it is timed
    std::vector<vx_trace_opts> cur(vols.size());
    for (size_t i = 0; i < vols.size(); i++) {
        Volume* V = vols[i];
        vx_trace_opts c{};
        std::lock_guard<std::mutex> lock(V->tune_mu);
        if (V->batch_tuned) c = V->tuned_batch;
        vx_trace_opts o{};
        o.mode = VX_MODE_PERSISTENT;
        o.block = c.block > 0 ? c.block : 256;
        o.refill = c.refill > 0 ? c.refill : kBatchRefill;
        o.burst = c.burst > 0 ? c.burst : kBatchBurst;
        cur[i] = o;
    }
    auto install = [&](const std::vector<vx_trace_opts>& asg) {
        for (size_t i = 0; i < vols.size(); i++) {
            std::lock_guard<std::mutex> lock(vols[i]->tune_mu);
            vols[i]->tuned_batch = asg[i];
            vols[i]->batch_tuned = true;
        }
    };
    auto timed = [&](const std::vector<vx_trace_opts>& asg, float* ms) {
        install(asg);
        int r = launch_batch(in, hit_layout, nullptr, st);
        if (r) return r;
        float best = 1e30f;
        for (int rep = 0; rep < 3; rep++) {
            cudaEventRecord(a, st);
            r = launch_batch(in, hit_layout, nullptr, st);
            if (r) return r;
            cudaEventRecord(b, st);
            cudaError_t e = cudaEventSynchronize(b);
            if (e) return cuda_fail(e, "autotune_batch");
            float t = 0.0f;
            cudaEventElapsedTime(&t, a, b);
            if (t < best) best = t;
        }
        *ms = best;
        return (int)VX_OK;
    };
    float cur_ms = 0.0f;
    int rc = timed(cur, &cur_ms);
    auto consider = [&](const std::vector<vx_trace_opts>& cand) {
        if (rc) return;
        float ms = 0.0f;
        rc = timed(cand, &ms);
        if (!rc && ms < cur_ms * 0.99f) { cur = cand; cur_ms = ms; }
    };
    // one knob of volume i (all volumes when i < 0) set to a value
    auto with = [&](int i, int knob, int value) {
        std::vector<vx_trace_opts> c = cur;
        for (size_t k = 0; k < c.size(); k++) {
            if (i >= 0 && (size_t)i != k) continue;
            if (knob == 0) c[k].refill = value;
            else if (knob == 1) c[k].burst = value;
            else c[k].block = value;
        }
        return c;
    };
    for (int round = 0; round < 2 && !rc; round++) {
        for (int r : {1, 2, 4, 8, 16}) consider(with(-1, 0, r));
        for (int bu : {4, 8, 16, 32}) consider(with(-1, 1, bu));
        for (int bl : {128, 256}) consider(with(-1, 2, bl));
    }
    for (int i = 0; i < (int)vols.size() && vols.size() > 1 && !rc; i++) {
        for (int r : {1, 2, 4, 8, 16}) consider(with(i, 0, r));
        for (int bu : {4, 8, 16, 32}) consider(with(i, 1, bu));
        for (int bl : {128, 256}) consider(with(i, 2, bl));
    }
    cudaEventDestroy(a);
    cudaEventDestroy(b);
    install(cur);  // the best assignment (also after an error: it was timed or is the start)
    if (rc) return rc;
    if (chosen)
        for (uint32_t i = 0; i < count; i++) {
            Volume& V = items[i].volume->v;
            std::lock_guard<std::mutex> lock(V.tune_mu);
            chosen[i] = V.batch_tuned ? V.tuned_batch : vx_trace_opts{};
        }
    return VX_OK;
}

extern "C" int vx_trace_host(vx_volume v, const vx_ray* rays_host, uint64_t n, void* hits_host, int32_t hit_layout,
                             const vx_trace_opts* opts, void* stream) {
    clear_error();
    int rc = check_trace_args(v, rays_host, n, hits_host, hit_layout);
    if (!rc) rc = check_opts(opts);
    if (rc || n == 0) return rc;
    if ((rc = check_ptrs(rays_host, hits_host, hit_layout))) return rc;
    if (!rays_host) return fail(VX_EINVAL, "rays is NULL");
    DeviceScope ds(v->v.device);
    if (ds.error()) return cuda_fail(ds.error(), "cudaSetDevice");
    const size_t hb = hit_bytes(hit_layout);
    Volume& V = v->v;
    return pipeline(V, n, stream, [&](uint64_t i0, uint64_t m, void* dr, void* dh, cudaStream_t st) {
        cudaError_t e = cudaMemcpyAsync(dr, rays_host + i0, m * sizeof(vx_ray), cudaMemcpyHostToDevice, st);
        if (e) return cuda_fail(e, "cudaMemcpyAsync (rays)");
        int r = launch_trace(V, (const vx_ray*)dr, m, dh, hit_layout, opts, st);
        if (r) return r;
        e = cudaMemcpyAsync((char*)hits_host + i0 * hb, dh, m * hb, cudaMemcpyDeviceToHost, st);
        if (e) return cuda_fail(e, "cudaMemcpyAsync (hits)");
        return (int)VX_OK;
    });
}

extern "C" int vx_trace_noalloc(vx_volume v, const vx_ray* rays, uint64_t n, void* hits, int32_t hit_layout,
                                void* stream) {
    clear_error();
    int rc = check_trace_args(v, rays, n, hits, hit_layout);
    if (rc) return rc;
    DeviceScope ds(v->v.device);
    if (ds.error()) return cuda_fail(ds.error(), "cudaSetDevice");
    return trace_noalloc(v->v, rays, n, hits, hit_layout, stream);
}

extern "C" int vx_raygen_pinhole(const vx_camera* cam, vx_ray* rays, void* stream) {
    clear_error();
    CameraParams cp;
    int rc = camera_params(cam, &cp);
    if (rc) return rc;
    if (!rays) return fail(VX_EINVAL, "rays is NULL");
    if (!aligned(rays, 16)) return fail(VX_EINVAL, "rays must be 16-byte aligned");
    return launch_raygen(cp, rays, stream);
}

extern "C" int vx_raygen_ao(const vx_ray* rays, const void* hits, uint64_t n, uint64_t seed, uint32_t spp, float eps,
                            float tmax, vx_ray* out, void* stream) {
    clear_error();
    if (n == 0 || spp == 0) return VX_OK;
    if (spp > 1024) return fail(VX_EINVAL, "spp must be at most 1024");
    if (!rays || !hits || !out) return fail(VX_EINVAL, "NULL array");
    if (!aligned(rays, 16) || !aligned(hits, 16) || !aligned(out, 16))
        return fail(VX_EINVAL, "rays, hits and out must be 16-byte aligned");
    if (!(eps >= 0.0f) || !(tmax > 0.0f)) return fail(VX_EINVAL, "eps must be >= 0 and tmax > 0");
    return launch_ao(rays, hits, n, seed, (int)spp, eps, tmax, out, stream);
}

extern "C" int vx_render(vx_volume v, const vx_camera* cam, void* hits, int32_t hit_layout, const vx_trace_opts* opts,
                         void* stream) {
    clear_error();
    CameraParams cp;
    int rc = camera_params(cam, &cp);
    if (rc) return rc;
    const uint64_t n = (uint64_t)cp.W * cp.H;
    rc = check_trace_args(v, nullptr, n, hits, hit_layout);
    if (!rc) rc = check_opts(opts);
    if (!rc) rc = check_ptrs(nullptr, hits, hit_layout);
    if (rc) return rc;
    DeviceScope ds(v->v.device);
    if (ds.error()) return cuda_fail(ds.error(), "cudaSetDevice");
    return launch_render(v->v, cp, 0, n, hits, hit_layout, opts, stream);
}

extern "C" int vx_render_views(vx_volume v, const vx_camera* cams, uint32_t count, void* const* hits,
                               int32_t hit_layout, const vx_trace_opts* opts, void* stream) {
    clear_error();
    if (count == 0) return VX_OK;
    if (!cams || !hits) return fail(VX_EINVAL, "cams or hits is NULL");
    if (count > 65536) return fail(VX_EINVAL, "at most 65536 views per call");
    int rc = check_opts(opts);
    if (rc) return rc;
    std::vector<CameraParams> cps(count);
    std::vector<uint64_t> i0(count, 0), n(count);
    for (uint32_t k = 0; k < count; k++) {
        rc = camera_params(&cams[k], &cps[k]);
        if (rc) return fail(rc, "view %u: %s", k, vx_last_error());
        n[k] = (uint64_t)cps[k].W * cps[k].H;
        rc = check_trace_args(v, nullptr, n[k], hits[k], hit_layout);
        if (!rc) rc = check_ptrs(nullptr, hits[k], hit_layout);
        if (rc) return fail(rc, "view %u: %s", k, vx_last_error());
    }
    DeviceScope ds(v->v.device);
    if (ds.error()) return cuda_fail(ds.error(), "cudaSetDevice");
    return launch_render_views(v->v, cps.data(), i0.data(), n.data(), hits, (int)count, hit_layout, opts, stream);
}

extern "C" int vx_render_host(vx_volume v, const vx_camera* cam, void* hits_host, int32_t hit_layout,
                              const vx_trace_opts* opts, void* stream) {
    clear_error();
    CameraParams cp;
    int rc = camera_params(cam, &cp);
    if (rc) return rc;
    const uint64_t n = (uint64_t)cp.W * cp.H;
    rc = check_trace_args(v, nullptr, n, hits_host, hit_layout);
    if (!rc) rc = check_opts(opts);
    if (!rc) rc = check_ptrs(nullptr, hits_host, hit_layout);
    if (rc) return rc;
    DeviceScope ds(v->v.device);
    if (ds.error()) return cuda_fail(ds.error(), "cudaSetDevice");
    const size_t hb = hit_bytes(hit_layout);
    Volume& V = v->v;
    return pipeline(V, n, stream, [&](uint64_t i0, uint64_t m, void*, void* dh, cudaStream_t st) {
        int r = launch_render(V, cp, i0, m, dh, hit_layout, opts, st);
        if (r) return r;
        cudaError_t e = cudaMemcpyAsync((char*)hits_host + i0 * hb, dh, m * hb, cudaMemcpyDeviceToHost, st);
        if (e) return cuda_fail(e, "cudaMemcpyAsync (hits)");
        return (int)VX_OK;
    });
}
