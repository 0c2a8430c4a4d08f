// noalloc.cu -- vx_trace_noalloc: the persistent trace for callers that must
// not allocate device memory.
//
// Some callers cannot call cudaMalloc at trace time: code running under a
// custom device-memory allocator that owns every byte of the GPU, real-time
// render loops that forbid allocation (and its implicit synchronisation)
// after start-up, or plug-ins hosted by an application that manages memory
// itself.  They pass their own ray and hit buffers; the only scratch this
// kernel needs, its ray-queue counter, lives in a small array of static
// device memory that the library reserves on every GPU that loads it, until
// the process exits.
//
// The scratch is shared by every call: each call zeroes the counter on its
// stream before the launch, and two calls whose kernels overlap on the GPU
// (different streams, or different threads) race on it and must not be
// issued.  The array is device memory; its name in host code is only a
// host-side stand-in, never a device address, so the host asks the runtime
// for the address (cudaGetSymbolAddress) once per device, with that device
// current, on the first call that uses the device.
#include <cuda_runtime.h>

#include <mutex>

#include "trace.cuh"
#include "vx_internal.hpp"

namespace vx {
namespace {

// 64 x 32-bit words; word 0 is the ray-queue counter.
constexpr int kNoAllocWords = 64;
static __device__ __align__(256) unsigned int g_noalloc_scratch[kNoAllocWords];

constexpr int kMaxDevices = 64;
std::mutex g_mu;
unsigned int* g_scratch_addr[kMaxDevices] = {};

// Device address of the scratch array on `dev` (which must be current).
int scratch_address(int dev, unsigned int** out) {
    if (dev < 0 || dev >= kMaxDevices) return fail(VX_EUNSUPPORTED, "device %d beyond the supported %d", dev, kMaxDevices);
    std::lock_guard<std::mutex> lock(g_mu);
    if (!g_scratch_addr[dev]) {
        void* p = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess)
            return fail(VX_ECUDA, "cudaGetSymbolAddress(scratch) on device %d: %s", dev, cudaGetErrorString(e));
        g_scratch_addr[dev] = static_cast<unsigned int*>(p);
    }
    *out = g_scratch_addr[dev];
    return VX_OK;
}

// The persistent trace with a 32-bit queue counter in the static scratch
// (same refill scheme as k_trace_persistent: a warp with >= `refill` idle
// lanes takes that many ray indices with one atomic).
template <int LAYOUT>
__global__ void __launch_bounds__(256) k_trace_noalloc(DynF f, const Img pool,
                                                       const float4* __restrict__ rays, uint32_t n,
                                                       void* __restrict__ hits, unsigned int* next, int refill,
                                                       int burst) {
    const unsigned lane = threadIdx.x & 31u;
    const unsigned lt_mask = (1u << lane) - 1u;
    Walker<false, DynF> w;  // node stack in the kernel's dynamic shared memory
    bool live = false;
    bool exhausted = false;  // warp-uniform
    uint32_t idx = 0;
    while (true) {
        const unsigned idle = __ballot_sync(0xffffffffu, !live);
        if (exhausted) {
            if (idle == 0xffffffffu) break;
        } else if (__popc(idle) >= refill) {
            const int leader = __ffs(idle) - 1;
            unsigned int base = 0;
            if ((int)lane == leader) base = atomicAdd(next, (unsigned int)__popc(idle));
            base = __shfl_sync(0xffffffffu, base, leader);
            if ((uint64_t)base + (uint64_t)__popc(idle) >= n) exhausted = true;
            if (!live) {
                idx = base + (uint32_t)__popc(idle & lt_mask);
                if ((uint64_t)base + __popc(idle & lt_mask) < n) {
                    HitRec h;
                    if (w.start(f, pool, load_ray(rays, idx), h)) store_hit<LAYOUT>(f, hits, idx, h);
                    else live = true;
                }
            }
            continue;
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

bool aligned(const void* p, size_t a) { return ((uintptr_t)p % a) == 0; }

}  // namespace

int trace_noalloc(const Volume& V, const vx_ray* rays, uint64_t n, void* hits, int layout, void* stream) {
    // The counter is 32 bits wide and every warp may add up to 32 past the
    // end, so the ray count stays below 2^32 - 2^24.
    if (n > VX_NOALLOC_MAX_RAYS)
        return fail(VX_EINVAL, "vx_trace_noalloc: %llu rays exceed the maximum of %llu (32-bit queue counter)",
                    (unsigned long long)n, (unsigned long long)VX_NOALLOC_MAX_RAYS);
    if (n == 0) return VX_OK;
    if (!rays || !aligned(rays, 16)) return fail(VX_EINVAL, "rays must be a non-NULL 16-byte aligned device array");
    if (!hits || !aligned(hits, layout == VX_HIT_FULL ? 16 : 8))
        return fail(VX_EINVAL, "hits must be a non-NULL device array aligned for the layout");
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e) return fail(VX_ECUDA, "cudaGetDevice: %s", cudaGetErrorString(e));
    unsigned int* next = nullptr;
    int rc = scratch_address(dev, &next);
    if (rc) return rc;
    int sms = 0, per_sm = 0;
    e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (e || sms < 1) return fail(VX_ECUDA, "SM count query: %s", cudaGetErrorString(e));
    const int block = 256;
    const size_t sm = stack_bytes(V.spec.fmt.J, block);
    e = layout == VX_HIT_FULL ? cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_trace_noalloc<0>, block, sm)
                              : cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_trace_noalloc<1>, block, sm);
    if (e) return fail(VX_ECUDA, "occupancy query: %s", cudaGetErrorString(e));
    if (per_sm < 1) per_sm = 1;
    uint64_t grid = (uint64_t)sms * per_sm;
    const uint64_t need = (n + block - 1) / block;
    if (grid > need) grid = need;
    cudaStream_t st = (cudaStream_t)stream;
    e = cudaMemsetAsync(next, 0, sizeof(unsigned int), st);  // the queue starts at zero on every call
    if (e) return fail(VX_ECUDA, "cudaMemsetAsync(scratch): %s", cudaGetErrorString(e));
    DynF f;
    f.p = V.spec.fmt;
    if (layout == VX_HIT_FULL)
        k_trace_noalloc<0><<<(unsigned)grid, block, sm, st>>>(f, Img{V.d_pool, V.packed, (uint32_t)V.pool_words, V.aligned}, reinterpret_cast<const float4*>(rays),
                                                              (uint32_t)n, hits, next, kDefaultRefill, kDefaultBurst);
    else
        k_trace_noalloc<1><<<(unsigned)grid, block, sm, st>>>(f, Img{V.d_pool, V.packed, (uint32_t)V.pool_words, V.aligned}, reinterpret_cast<const float4*>(rays),
                                                              (uint32_t)n, hits, next, kDefaultRefill, kDefaultBurst);
    e = cudaGetLastError();
    if (e) return fail(VX_ECUDA, "vx_trace_noalloc launch: %s", cudaGetErrorString(e));
    return VX_OK;
}

}  // namespace vx
