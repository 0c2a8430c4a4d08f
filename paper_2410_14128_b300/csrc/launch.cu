// launch.cu -- kernel registry, the run-time-described kernel set, camera set-up
// and the pinhole ray generator.
#include <math.h>
#include <string.h>

#include <algorithm>
#include <mutex>
#include <vector>

#include "trace.cuh"
#include "vx_internal.hpp"

namespace vx {

namespace {
std::vector<const KernelSet*>& registry() {
    static std::vector<const KernelSet*> r;
    return r;
}
const KernelSet g_generic = {"*",
                             false,
                             FmtParams{},
                             &Launch<DynF>::trace,
                             &Launch<DynF>::render,
                             &Launch<DynF>::trace_count,
                             &Launch<DynF>::trace_persistent,
                             &Launch<DynF>::trace_batch,
                             &Launch<DynF>::resident_blocks,
                             &Launch<DynF>::render_persistent};

CamDev to_dev(const CameraParams& c) {
    CamDev d;
    for (int i = 0; i < 3; i++) { d.eye[i] = c.eye[i]; d.f[i] = c.f[i]; d.r[i] = c.r[i]; d.u[i] = c.u[i]; }
    d.tha = c.tha; d.th = c.th; d.W = c.W; d.H = c.H;
    return d;
}

Img img_of(const Volume& v) { return Img{v.d_pool, v.packed, (uint32_t)v.pool_words, v.aligned}; }

}  // namespace

// Image words a persistent trace stages for smem_top = k: the prefix holding
// the top k node levels of a relocated image, at the largest k <= the one
// asked for whose prefix fits kTopSmemMaxWords; 0 for none.
uint32_t stage_words(const Volume& v, int k) {
    if (!v.aligned || k <= 0) return 0;
    if (k > kStageLevels) k = kStageLevels;
    for (; k > 0; k--)
        if (v.stage_end[k] <= kTopSmemMaxWords) return v.stage_end[k];
    return 0;
}

namespace {

// Default block sizes: 256 for persistent kernels (4 resident blocks per
// SM), 64 for the plain trace kernel, whose blocks each run until their
// slowest ray ends: smaller blocks free their SM share sooner (plain traces
// of 1080p views and of incoherent rays ran 5-23% faster at 64 than at 256).
int pick_block(const vx_trace_opts* o, int mode = VX_MODE_PERSISTENT) {
    if (o && o->block > 0) return o->block;
    return mode == VX_MODE_PLAIN ? 64 : 256;
}

__global__ void __launch_bounds__(256) k_raygen(CamDev cam, float4* __restrict__ rays) {
    const uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= (uint64_t)cam.W * cam.H) return;
    const RayIn r = pinhole_ray(cam, (uint32_t)(i % cam.W), (uint32_t)(i / cam.W));
    __stcs(rays + 2 * i, make_float4(r.o[0], r.o[1], r.o[2], r.tmin));
    __stcs(rays + 2 * i + 1, make_float4(r.d[0], r.d[1], r.d[2], r.tmax));
}
// Ambient-occlusion rays from primary hits: cosine-weighted about the
// outward normal of the entered face (Malley's method: a uniform point on the
// unit disk lifted to the hemisphere), two uniforms per ray from SplitMix64
// (Steele, Lea & Flood 2014) of the counter (i * spp + k) * 2 + {0, 1} mixed
// with the seed, top 24 bits.  The origin is the hit point moved eps along
// the normal.  Misses and hits with no entry face give the empty ray (all
// zero), which every trace reports as a miss.
__host__ __device__ __forceinline__ uint64_t sm64(uint64_t x) {
    x += 0x9E3779B97F4A7C15ull;
    x = (x ^ (x >> 30)) * 0xBF58476D1CE4E5B9ull;
    x = (x ^ (x >> 27)) * 0x94D049BB133111EBull;
    return x ^ (x >> 31);
}

__global__ void __launch_bounds__(256) k_ao_rays(const float4* __restrict__ rays, const uint4* __restrict__ hits,
                                                 uint64_t n, uint64_t seed_mix, int spp, float eps, float tmax,
                                                 float4* __restrict__ out) {
    const uint64_t j = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= n * (uint64_t)spp) return;
    const uint64_t i = j / (uint64_t)spp;
    const uint4 h = __ldg(hits + i);
    const uint32_t status = h.w >> 24, face = (h.w >> 16) & 0xFFu;
    float4 a = make_float4(0.f, 0.f, 0.f, 0.f), b = make_float4(0.f, 0.f, 0.f, 0.f);
    if (status == ST_HIT && face != 0) {
        const int ax = (int)(face - 1) / 2;
        const float sign = ((face - 1) & 1u) ? 1.0f : -1.0f;
        const uint64_t c = j * 2u;
        const float u1 = (float)(sm64(seed_mix ^ c) >> 40) * 0x1.0p-24f;
        const float u2 = (float)(sm64(seed_mix ^ (c + 1)) >> 40) * 0x1.0p-24f;
        const float r = sqrtf(u1);
        float sp, cp;
        sincospif(2.0f * u2, &sp, &cp);
        const float lz = sqrtf(fmaxf(1.0f - u1, 0.0f));
        float d[3] = {0.f, 0.f, 0.f};
        const int a1 = ax == 2 ? 0 : ax + 1, a2 = ax == 0 ? 2 : ax - 1;
#pragma unroll
        for (int q = 0; q < 3; q++) d[q] = q == a1 ? r * cp : (q == a2 ? r * sp : (q == ax ? sign * lz : 0.f));
        const float4 ra = __ldg(rays + 2 * i), rb = __ldg(rays + 2 * i + 1);
        const float t = __uint_as_float(h.x);
        float p[3] = {fmaf(t, rb.x, ra.x), fmaf(t, rb.y, ra.y), fmaf(t, rb.z, ra.z)};
#pragma unroll
        for (int q = 0; q < 3; q++)
            if (q == ax) p[q] += sign * eps;
        a = make_float4(p[0], p[1], p[2], 0.0f);
        b = make_float4(d[0], d[1], d[2], tmax);
    }
    __stcs(out + 2 * j, a);
    __stcs(out + 2 * j + 1, b);
}
}  // namespace

void register_kernel_set(const KernelSet* ks) { registry().push_back(ks); }

unsigned long long* Volume::queue_counter(void* stream) const {
    if (!d_queue) return nullptr;
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    if (cudaStreamIsCapturing((cudaStream_t)stream, &cs) != cudaSuccess) return nullptr;
    if (cs == cudaStreamCaptureStatusActive) {
        const uint32_t k = captured_slot.fetch_add(1, std::memory_order_relaxed);
        if (k >= (uint32_t)kQueueCaptured) return nullptr;
        return d_queue + kQueueRing + k;
    }
    return d_queue + (queue_slot.fetch_add(1, std::memory_order_relaxed) % kQueueRing);
}

void prefer_carveout(const void* kernel, size_t smem_per_block, int block) {
    static std::mutex mu;
    static std::vector<std::pair<std::pair<const void*, int>, int>> done;  // ((kernel, device), percent) set
    int dev = 0;
    if (cudaGetDevice(&dev)) return;
    const int blocks = block > 0 ? (1024 + block - 1) / block : 1;
    const size_t need = (size_t)blocks * (smem_per_block + 1024);  // 1 KiB per block is reserved
    const size_t max_smem = 228u * 1024u;
    int pct = (int)((need * 100 + max_smem - 1) / max_smem);
    if (pct > 100) pct = 100;
    std::lock_guard<std::mutex> lock(mu);
    for (auto& d : done)
        if (d.first.first == kernel && d.first.second == dev) {
            if (d.second == pct) return;
            d.second = pct;
            cudaFuncSetAttribute(kernel, cudaFuncAttributePreferredSharedMemoryCarveout, pct);
            return;
        }
    done.emplace_back(std::make_pair(kernel, dev), pct);
    cudaFuncSetAttribute(kernel, cudaFuncAttributePreferredSharedMemoryCarveout, pct);
}

int launch_ao(const vx_ray* rays, const void* hits, uint64_t n, uint64_t seed, int spp, float eps, float tmax,
              vx_ray* out, void* stream) {
    const uint64_t m = n * (uint64_t)spp;
    if (m == 0) return VX_OK;
    k_ao_rays<<<(unsigned)((m + 255) / 256), 256, 0, (cudaStream_t)stream>>>(
        reinterpret_cast<const float4*>(rays), reinterpret_cast<const uint4*>(hits), n, sm64(seed), spp, eps, tmax,
        reinterpret_cast<float4*>(out));
    cudaError_t e = cudaGetLastError();
    if (e) return fail(VX_ECUDA, "ao launch: %s", cudaGetErrorString(e));
    return VX_OK;
}

const KernelSet* find_kernels(const std::string& spec) {
    for (const KernelSet* k : registry())
        if (spec == k->spec) return k;
    return nullptr;
}

const KernelSet* generic_kernels() { return &g_generic; }

std::vector<const KernelSet*> registered_kernel_sets() { return registry(); }

const char* kernel_set_spec(const KernelSet* k) { return k->spec; }

bool kernel_set_specialized(const KernelSet* k) { return k && k->specialized; }

static bool same_params(const FmtParams& a, const FmtParams& b) { return memcmp(&a, &b, sizeof(FmtParams)) == 0; }

const KernelSet* kernels_for(const Spec& sp) {
    const KernelSet* k = find_kernels(sp.canonical);
    if (k && same_params(k->params, sp.fmt)) return k;
    return generic_kernels();
}

int launch_trace(const Volume& v, const vx_ray* rays, uint64_t n, void* hits, int layout, const vx_trace_opts* o,
                 void* stream) {
    // VX_MODE_AUTO takes the autotuned options when the volume has them.
    vx_trace_opts tuned;
    if (!o || o->mode == VX_MODE_AUTO) {
        Volume& mv = const_cast<Volume&>(v);
        std::lock_guard<std::mutex> lock(mv.tune_mu);
        if (mv.tuned) {
            tuned = mv.tuned_opts;
            o = &tuned;
        }
    }
    const int mode = (o && o->mode != VX_MODE_AUTO) ? o->mode : VX_MODE_PERSISTENT;
    const int block = pick_block(o, mode);
    const int sort = o ? o->sort_cell_log2 : 0;
    const int restart = o ? o->restart : 0;
    // the walker's resume mode: full node stack, restarting traversal, or a short stack of depth D
    const int stack = restart ? -1 : (o ? o->short_stack : 0);
    cudaStream_t st = (cudaStream_t)stream;
    // Optional coherence sort: scratch from the stream-ordered pool, freed
    // on the same stream after the trace.  The trace then runs on the sorted
    // copy of the rays into sorted hits, which a gather puts back in order.
    void* scratch = nullptr;
    SortedRays sorted;
    const vx_ray* trays = rays;
    void* thits = hits;
    if (sort > 0) {
        const uint32_t hb = layout == VX_HIT_FULL ? 16u : 8u;
        const uint64_t bytes = sort_scratch_bytes(v.spec.ldim, sort, n, hb, nullptr);
        cudaError_t ce = cudaMallocAsync(&scratch, bytes, st);
        if (ce) return fail(ce == cudaErrorMemoryAllocation ? VX_ENOMEM : VX_ECUDA, "sort scratch: %s",
                            cudaGetErrorString(ce));
        int rc = sort_rays(v.spec.ldim, sort, rays, n, hb, scratch, &sorted, st);
        if (rc) {
            cudaFreeAsync(scratch, st);
            return rc;
        }
        trays = sorted.rays;
        thits = sorted.hits;
    }
    int e;
    if (mode == VX_MODE_PERSISTENT) {
        unsigned long long* next = v.queue_counter(st);
        if (!next) {
            if (scratch) cudaFreeAsync(scratch, st);
            return fail(VX_EUNSUPPORTED, "no queue counter for the persistent kernel (at most %d captured "
                        "persistent launches per volume)", kQueueCaptured);
        }
        const int refill = (o && o->refill > 0) ? o->refill : kDefaultRefill;
        const int burst = (o && o->burst > 0) ? o->burst : kDefaultBurst;
        const int bps = o ? o->blocks_per_sm : 0;
        const uint32_t stage = stage_words(v, o ? o->smem_top : 0);
        e = v.kernels->trace_persistent(v.spec.fmt, img_of(v), reinterpret_cast<const float4*>(trays), n, thits,
                                        layout, block, bps, refill, burst, stack, stage, st, next);
    } else {
        e = v.kernels->trace(v.spec.fmt, img_of(v), reinterpret_cast<const float4*>(trays), n, thits, layout,
                             block, stack, st);
    }
    if (!e && scratch) {
        const int rc = unsort_hits(sorted, n, hits, layout, st);
        if (rc) {
            cudaFreeAsync(scratch, st);
            return rc;
        }
    }
    if (scratch) cudaFreeAsync(scratch, st);
    if (e) return fail(VX_ECUDA, "trace launch failed: %s", cudaGetErrorString((cudaError_t)e));
    return VX_OK;
}

int launch_trace_count(const Volume& v, const vx_ray* rays, uint64_t n, void* hits, int layout,
                       const vx_trace_opts* o, void* stream, unsigned long long* counters, uint32_t* sectors) {
    const int block = pick_block(o);
    const int restart = o ? o->restart : 0;
    int e = v.kernels->trace_count(v.spec.fmt, img_of(v), reinterpret_cast<const float4*>(rays), n, hits, layout,
                                   block, restart, (cudaStream_t)stream, counters, sectors);
    if (e) return fail(VX_ECUDA, "trace launch failed: %s", cudaGetErrorString((cudaError_t)e));
    return VX_OK;
}

int launch_render(const Volume& v, const CameraParams& cp, uint64_t i0, uint64_t n, void* hits, int layout,
                  const vx_trace_opts* o, void* stream) {
    return launch_render_views(v, &cp, &i0, &n, &hits, 1, layout, o, stream);
}

int launch_render_views(const Volume& v, const CameraParams* cps, const uint64_t* i0, const uint64_t* n,
                        void* const* hits, int count, int layout, const vx_trace_opts* o, void* stream) {
    const int mode = (o && o->mode != VX_MODE_AUTO) ? o->mode : VX_MODE_PLAIN;  // coherent views: plain
    // the tiled render kernel defaults to blocks of 128 (4 tiles of 8 x 4
    // pixels): 2% faster than 256 on the 1080p benchmark views
    const int block = (o && o->block > 0) ? o->block : (mode == VX_MODE_PERSISTENT ? pick_block(o) : 128);
    int e = 0;
    if (mode == VX_MODE_PERSISTENT) {
        // one persistent launch per view
        const int refill = (o && o->refill > 0) ? o->refill : kDefaultRefill;
        const int burst = (o && o->burst > 0) ? o->burst : kDefaultBurst;
        for (int k = 0; k < count && !e; k++) {
            if (n[k] == 0) continue;
            unsigned long long* next = v.queue_counter(stream);
            if (!next)
                return fail(VX_EUNSUPPORTED, "no queue counter for the persistent kernel (at most %d captured "
                            "persistent launches per volume)", kQueueCaptured);
            e = v.kernels->render_persistent(v.spec.fmt, img_of(v), to_dev(cps[k]), i0[k], n[k], hits[k], layout,
                                             block, refill, burst, (cudaStream_t)stream, next);
        }
    } else {
        std::vector<CamDev> cams((size_t)count);
        for (int k = 0; k < count; k++) cams[(size_t)k] = to_dev(cps[k]);
        e = v.kernels->render(v.spec.fmt, img_of(v), cams.data(), i0, n, hits, count, layout, block,
                              (cudaStream_t)stream);
    }
    if (e) return fail(VX_ECUDA, "render launch failed: %s", cudaGetErrorString((cudaError_t)e));
    return VX_OK;
}

// ---------------------------------------------------------------------------
// Batched tracing: group the sets by format, one persistent launch per group
// (sub-groups of kBatchMax sets), all launches concurrent on forked streams,
// the SMs shared in proportion to each launch's rays.
// ---------------------------------------------------------------------------
namespace {
constexpr int kForkStreams = 8;
struct DevStreams {
    bool ready = false;
    cudaStream_t s[kForkStreams];
    cudaEvent_t fork;
    cudaEvent_t join[kForkStreams];
};
std::mutex g_fork_mu;
DevStreams g_fork[64];
}  // namespace

int launch_batch(const std::vector<BatchItemIn>& items, int layout, const vx_trace_opts* o, void* stream,
                 void** events, uint32_t n_events, uint32_t* groups) {
    cudaStream_t st = (cudaStream_t)stream;
    int dev = 0, sms = 0;
    cudaError_t ce = cudaGetDevice(&dev);
    if (ce) return fail(VX_ECUDA, "cudaGetDevice: %s", cudaGetErrorString(ce));
    if (dev >= 64) return fail(VX_EUNSUPPORTED, "device %d", dev);
    ce = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (ce || sms < 1) return fail(VX_ECUDA, "SM count: %s", cudaGetErrorString(ce));
    if (groups) *groups = 0;
    // group by (kernel set, format parameters)
    struct Sub {
        const KernelSet* ks;
        const Volume* v0;
        BatchDesc d;
    };
    std::vector<Sub> subs;
    for (const BatchItemIn& it : items) {
        if (it.n == 0) continue;
        Sub* g = nullptr;
        for (Sub& s2 : subs)
            if (s2.ks == it.v->kernels && same_params(s2.v0->spec.fmt, it.v->spec.fmt) &&
                s2.d.packed == it.v->packed && s2.d.aligned == it.v->aligned && s2.d.count < kBatchMax) {
                g = &s2;
                break;
            }
        if (!g) {
            subs.push_back(Sub{it.v->kernels, it.v, BatchDesc{}});
            g = &subs.back();
            g->d.count = 0;
            g->d.packed = it.v->packed;
            g->d.aligned = it.v->aligned;
            g->d.start[0] = 0;
        }
        const uint32_t k = g->d.count++;
        g->d.pool[k] = it.v->d_pool;
        g->d.rays[k] = reinterpret_cast<const float4*>(it.rays);
        g->d.hits[k] = it.hits;
        g->d.start[k + 1] = g->d.start[k] + it.n;
    }
    if (subs.empty()) return VX_OK;
    // Options of each group: explicit ones, else the block, refill and burst
    // vx_autotune_batch chose for its volume, else the batched defaults.
    // (A volume's vx_autotune options are tuned on one launch alone and did
    // not carry over: 2005-2085 Mrays/s over runs against 2075 for the
    // defaults.)
    const int nsub = (int)subs.size();
    std::vector<vx_trace_opts> gopts(nsub);
    for (int i = 0; i < nsub; i++) {
        vx_trace_opts def{};
        if (!o || o->mode == VX_MODE_AUTO) {
            Volume& mv = const_cast<Volume&>(*subs[i].v0);
            std::lock_guard<std::mutex> lock(mv.tune_mu);
            if (mv.batch_tuned) def = mv.tuned_batch;
        } else {
            def = *o;
        }
        if (def.block <= 0) def.block = 256;
        if (def.refill <= 0) def.refill = kBatchRefill;
        if (def.burst <= 0) def.burst = kBatchBurst;
        gopts[i] = def;
    }

    std::lock_guard<std::mutex> lock(g_fork_mu);
    DevStreams& F = g_fork[dev];
    if (!F.ready) {
        for (int i = 0; i < kForkStreams; i++) {
            cudaError_t e = cudaStreamCreateWithFlags(&F.s[i], cudaStreamNonBlocking);
            if (!e) e = cudaEventCreateWithFlags(&F.join[i], cudaEventDisableTiming);
            if (e) return fail(VX_ECUDA, "batch streams: %s", cudaGetErrorString(e));
        }
        cudaError_t e = cudaEventCreateWithFlags(&F.fork, cudaEventDisableTiming);
        if (e) return fail(VX_ECUDA, "batch events: %s", cudaGetErrorString(e));
        F.ready = true;
    }
    // Grid of every group, decided before anything is enqueued: a failure
    // here leaves no forked stream behind.
    // Every launch gets a full GPU's worth of resident blocks: the launches
    // run one after another in effect, each draining its queue with all SMs,
    // and the next one's blocks start as the previous one's retire (separate
    // streams), so no SM waits for a slower group.
    std::vector<int> grids(nsub);
    std::vector<unsigned long long*> nexts(nsub);
    for (int i = 0; i < nsub; i++) {
        const Sub& g = subs[i];
        nexts[i] = g.v0->queue_counter(st);  // the fork streams inherit the caller's capture state
        if (!nexts[i])
            return fail(VX_EUNSUPPORTED, "no queue counter for the batched kernel (at most %d captured "
                        "persistent launches per volume)", kQueueCaptured);
        const int block = gopts[i].block;
        int per_sm = 1;
        int rc = g.ks->resident_blocks(g.v0->spec.fmt, layout, block, &per_sm);
        if (rc) return fail(VX_ECUDA, "occupancy: %s", cudaGetErrorString((cudaError_t)rc));
        const uint64_t n = g.d.start[g.d.count];
        uint64_t grid = (uint64_t)sms * per_sm;
        const uint64_t need = (n + block - 1) / block;
        if (grid > need) grid = need;
        grids[i] = grid < 1 ? 1 : (int)grid;
    }
    cudaError_t e = cudaEventRecord(F.fork, st);
    if (e) return fail(VX_ECUDA, "batch fork: %s", cudaGetErrorString(e));
    const int nfork = nsub < kForkStreams ? nsub : kForkStreams;
    int forked = 0;
    for (; forked < nfork; forked++) {
        e = cudaStreamWaitEvent(F.s[forked], F.fork, 0);
        if (e) break;
    }
    int rc = e ? fail(VX_ECUDA, "batch fork: %s", cudaGetErrorString(e)) : VX_OK;
    // Timing events: inside a stream capture a record needs
    // cudaEventRecordExternal to become an event node of the graph (a plain
    // record there is only a dependency edge); outside a capture that flag is
    // not allowed.
    unsigned int rec_flags = cudaEventRecordDefault;
    if (events && !rc) {
        cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
        e = cudaStreamIsCapturing(st, &cs);
        if (e) rc = fail(VX_ECUDA, "batch capture state: %s", cudaGetErrorString(e));
        else if (cs == cudaStreamCaptureStatusActive) rec_flags = cudaEventRecordExternal;
    }
    for (int i = 0; i < nsub && !rc; i++) {
        Sub& g = subs[i];
        cudaStream_t fs = F.s[i % kForkStreams];
        const bool timed = events && (uint32_t)(2 * i + 1) < n_events;
        if (timed && (e = cudaEventRecordWithFlags((cudaEvent_t)events[2 * i], fs, rec_flags))) {
            rc = fail(VX_ECUDA, "batch timing event: %s", cudaGetErrorString(e));
            break;
        }
        const vx_trace_opts& go = gopts[i];
        int lr = g.ks->trace_batch(g.v0->spec.fmt, g.d, layout, go.block, grids[i], go.refill, go.burst, fs, nexts[i]);
        if (lr) {
            rc = fail(VX_ECUDA, "batch launch: %s", cudaGetErrorString((cudaError_t)lr));
            break;
        }
        if (timed && (e = cudaEventRecordWithFlags((cudaEvent_t)events[2 * i + 1], fs, rec_flags))) {
            rc = fail(VX_ECUDA, "batch timing event: %s", cudaGetErrorString(e));
            break;
        }
        if (groups) *groups = (uint32_t)(i + 1);
    }
    // Join every forked stream back into the caller's stream, on success and
    // on failure alike: a stream left forked would invalidate a capture in
    // progress and keep waiting on the caller's work.
    for (int i = 0; i < forked; i++) {
        cudaError_t j1 = cudaEventRecord(F.join[i], F.s[i]);
        cudaError_t j2 = j1 ? j1 : cudaStreamWaitEvent(st, F.join[i], 0);
        if (j2 && !rc) rc = fail(VX_ECUDA, "batch join: %s", cudaGetErrorString(j2));
    }
    if (rc) return rc;
    e = cudaGetLastError();
    if (e) return fail(VX_ECUDA, "batch: %s", cudaGetErrorString(e));
    return VX_OK;
}

// ---------------------------------------------------------------------------
// Batched tracing from host memory: the rays of all sets stream through the
// device in waves of at most kWaveRays rays (a set larger than the room left
// in a wave is split across waves).  Wave w uses staging buffer w % kWaves
// and stream w % kWaves: its uploads, its batched kernels (launch_batch,
// forked and joined on that stream) and its downloads are ordered on that
// stream, so the upload of one wave, the kernels of another and the download
// of a third run at once on the two copy engines and the SMs, and a buffer is
// reused only after the wave that last used it has been copied back.
// ---------------------------------------------------------------------------
namespace {
// 2^21 rays per wave (64 MiB of rays, 32 MiB of full hits per buffer), four
// waves in flight: the 2048^3 batched workload from pinned memory ran at
// 63.3 ms a step, against 64.5 ms with 2^22 x 3 and 68.6 ms with 2^20 x 6
constexpr uint64_t kWaveRays = 1ull << 21;
constexpr int kWaves = 4;
struct WaveStaging {
    std::mutex mu;
    bool ready = false;
    void* d_rays[kWaves] = {};
    void* d_hits[kWaves] = {};
    cudaStream_t s[kWaves] = {};
    cudaEvent_t start = nullptr;
};
WaveStaging g_waves[64];

int wave_staging(WaveStaging& W) {
    if (W.ready) return VX_OK;
    cudaError_t e = cudaEventCreateWithFlags(&W.start, cudaEventDisableTiming);
    for (int b = 0; b < kWaves && !e; b++) {
        e = cudaMalloc(&W.d_rays[b], kWaveRays * sizeof(vx_ray));
        if (!e) e = cudaMalloc(&W.d_hits[b], kWaveRays * 16u);
        if (!e) e = cudaStreamCreateWithFlags(&W.s[b], cudaStreamNonBlocking);
    }
    if (e) {
        for (int b = 0; b < kWaves; b++) {
            if (W.d_rays[b]) cudaFree(W.d_rays[b]);
            if (W.d_hits[b]) cudaFree(W.d_hits[b]);
            if (W.s[b]) cudaStreamDestroy(W.s[b]);
            W.d_rays[b] = W.d_hits[b] = nullptr;
            W.s[b] = nullptr;
        }
        if (W.start) cudaEventDestroy(W.start);
        W.start = nullptr;
        return fail(e == cudaErrorMemoryAllocation ? VX_ENOMEM : VX_ECUDA, "wave staging: %s",
                    cudaGetErrorString(e));
    }
    W.ready = true;
    return VX_OK;
}
}  // namespace

int launch_batch_host(const std::vector<BatchItemIn>& items, int layout, const vx_trace_opts* o, void* stream) {
    int dev = 0;
    cudaError_t ce = cudaGetDevice(&dev);
    if (ce) return fail(VX_ECUDA, "cudaGetDevice: %s", cudaGetErrorString(ce));
    if (dev < 0 || dev >= 64) return fail(VX_EUNSUPPORTED, "device index %d above 63", dev);
    // the call waits for its copies, which a stream capture cannot hold
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    ce = cudaStreamIsCapturing((cudaStream_t)stream, &cs);
    if (ce) return fail(VX_ECUDA, "cudaStreamIsCapturing: %s", cudaGetErrorString(ce));
    if (cs != cudaStreamCaptureStatusNone)
        return fail(VX_EUNSUPPORTED, "tracing from host memory waits for its copies: not on a capturing stream");
    WaveStaging& W = g_waves[dev];
    std::lock_guard<std::mutex> lock(W.mu);
    int rc = wave_staging(W);
    if (rc) return rc;
    const size_t hb = layout == VX_HIT_FULL ? 16u : 8u;
    // the waves start after the caller's earlier work on its stream
    ce = cudaEventRecord(W.start, (cudaStream_t)stream);
    for (int b = 0; b < kWaves && !ce; b++) ce = cudaStreamWaitEvent(W.s[b], W.start, 0);
    if (ce) return fail(VX_ECUDA, "wave start: %s", cudaGetErrorString(ce));
    struct Slice {
        size_t item;
        uint64_t off, m, at;  // rays [off, off + m) of the item at ray `at` of the wave buffer
    };
    std::vector<Slice> slices;
    std::vector<BatchItemIn> dev_items;
    size_t item = 0;
    uint64_t off = 0;
    for (uint64_t w = 0; item < items.size() && !rc; w++) {
        const int b = (int)(w % kWaves);
        cudaStream_t s = W.s[b];
        vx_ray* dr = (vx_ray*)W.d_rays[b];
        char* dh = (char*)W.d_hits[b];
        slices.clear();
        dev_items.clear();
        uint64_t fill = 0;
        while (item < items.size() && fill < kWaveRays) {
            const uint64_t m = std::min(items[item].n - off, kWaveRays - fill);
            if (m > 0) slices.push_back(Slice{item, off, m, fill});
            fill += m;
            off += m;
            if (off >= items[item].n) {
                item++;
                off = 0;
            }
        }
        for (const Slice& sl : slices) {
            ce = cudaMemcpyAsync(dr + sl.at, items[sl.item].rays + sl.off, sl.m * sizeof(vx_ray),
                                 cudaMemcpyHostToDevice, s);
            if (ce) break;
            dev_items.push_back(BatchItemIn{items[sl.item].v, dr + sl.at, sl.m, dh + sl.at * hb});
        }
        if (ce) {
            rc = fail(VX_ECUDA, "cudaMemcpyAsync (rays): %s", cudaGetErrorString(ce));
            break;
        }
        if (!dev_items.empty()) rc = launch_batch(dev_items, layout, o, s);
        if (rc) break;
        for (const Slice& sl : slices) {
            ce = cudaMemcpyAsync((char*)items[sl.item].hits + sl.off * hb, dh + sl.at * hb, sl.m * hb,
                                 cudaMemcpyDeviceToHost, s);
            if (ce) break;
        }
        if (ce) rc = fail(VX_ECUDA, "cudaMemcpyAsync (hits): %s", cudaGetErrorString(ce));
    }
    // nothing may still read or write the caller's memory after the return
    for (int b = 0; b < kWaves; b++) {
        ce = cudaStreamSynchronize(W.s[b]);
        if (ce && !rc) rc = fail(VX_ECUDA, "batch from host memory: %s", cudaGetErrorString(ce));
    }
    return rc;
}


int launch_raygen(const CameraParams& cp, vx_ray* rays, void* stream) {
    const uint64_t n = (uint64_t)cp.W * cp.H;
    if (n == 0) return VX_OK;
    k_raygen<<<(unsigned)((n + 255) / 256), 256, 0, (cudaStream_t)stream>>>(to_dev(cp), reinterpret_cast<float4*>(rays));
    cudaError_t e = cudaGetLastError();
    if (e) return fail(VX_ECUDA, "raygen launch failed: %s", cudaGetErrorString(e));
    return VX_OK;
}

// Camera basis in FP64 on the host, handed to the kernels in FP32.
int camera_params(const vx_camera* cam, CameraParams* out) {
    if (!cam) return fail(VX_EINVAL, "camera is NULL");
    if (cam->width == 0 || cam->height == 0) return fail(VX_EINVAL, "camera has an empty image");
    if (!(cam->vfov_deg > 0.0 && cam->vfov_deg < 180.0)) return fail(VX_EINVAL, "vfov must be in (0, 180)");
    double f[3], r[3], u[3];
    for (int i = 0; i < 3; i++) f[i] = cam->look[i] - cam->eye[i];
    double lf = sqrt(f[0] * f[0] + f[1] * f[1] + f[2] * f[2]);
    if (!(lf > 0.0)) return fail(VX_EINVAL, "camera eye and look coincide");
    for (int i = 0; i < 3; i++) f[i] /= lf;
    const double* up = cam->up;
    r[0] = f[1] * up[2] - f[2] * up[1];
    r[1] = f[2] * up[0] - f[0] * up[2];
    r[2] = f[0] * up[1] - f[1] * up[0];
    double lr = sqrt(r[0] * r[0] + r[1] * r[1] + r[2] * r[2]);
    if (!(lr > 0.0)) return fail(VX_EINVAL, "camera up is parallel to the view direction");
    for (int i = 0; i < 3; i++) r[i] /= lr;
    u[0] = r[1] * f[2] - r[2] * f[1];
    u[1] = r[2] * f[0] - r[0] * f[2];
    u[2] = r[0] * f[1] - r[1] * f[0];
    const double th = tan(cam->vfov_deg * 3.14159265358979323846 / 360.0);
    for (int i = 0; i < 3; i++) {
        out->eye[i] = (float)cam->eye[i];
        out->f[i] = (float)f[i];
        out->r[i] = (float)r[i];
        out->u[i] = (float)u[i];
    }
    out->th = (float)th;
    out->tha = (float)(th * (double)cam->width / (double)cam->height);
    out->W = cam->width;
    out->H = cam->height;
    return VX_OK;
}

}  // namespace vx
