// sort.cu -- ray sorting for coherence before tracing.
//
// Key of a ray = direction octant (3 bits) above the Morton code (x lowest,
// Fig. 5 order) of its origin's cell of side 2^g voxels, the origin clamped
// into the grid.  The code keeps at most 5 bits per axis (2^18 bins in all):
// when an axis has more than 5 bits of cells, the key takes its 5 coarsest
// ones, i.e. cells of side 2^(log2 dim - 5) on that axis.  Rays with equal keys start close together and head the
// same way, so a warp that traces consecutive sorted rays reads the same
// nodes and takes similar paths.  A counting sort by key (histogram,
// exclusive scan, scatter) gives each ray its position in key order; the
// scatter also copies the rays there (coalesced reads, whole 32-byte sectors
// written), the trace runs on that sorted copy writing sorted hits in order,
// and a gather puts each hit back at its ray's index (random reads of the
// sorted hits, which the L2 still holds, and coalesced writes).  So neither
// the trace's ray reads nor its hit writes touch scattered partial sectors.
#include <cuda_runtime.h>

#include "trace.cuh"
#include "vx_internal.hpp"

namespace vx {
namespace {

struct KeyParams {
    int ld[3];
    int g;      // cell side 2^g
    int kb[3];  // Morton bits per axis: min(max(ld - g, 0), 5)
    int sh[3];  // shift of a voxel coordinate to its key cell: ld - kb (= g unless capped)
    int mbits;  // kb[0] + kb[1] + kb[2]
};

__device__ __forceinline__ uint32_t ray_key(const float4 a, const float4 b, const KeyParams& k) {
    const float o[3] = {a.x, a.y, a.z};
    const float d[3] = {b.x, b.y, b.z};
    uint32_t cell[3];
#pragma unroll
    for (int i = 0; i < 3; i++) {
        const float n = (float)(1 << k.ld[i]);
        float v = fminf(fmaxf(o[i], 0.0f), n - 1.0f);  // NaN -> 0
        if (!(v == v)) v = 0.0f;
        cell[i] = ((uint32_t)v) >> k.sh[i];
    }
    uint32_t m = 0;
    int bit = 0;
#pragma unroll
    for (int b2 = 0; b2 < 10; b2++)
#pragma unroll
        for (int i = 0; i < 3; i++)
            if (b2 < k.kb[i]) m |= ((cell[i] >> b2) & 1u) << bit++;
    const uint32_t oct = (d[0] < 0.0f ? 1u : 0u) | (d[1] < 0.0f ? 2u : 0u) | (d[2] < 0.0f ? 4u : 0u);
    return (oct << k.mbits) | m;
}

// Key of each ray, and its rank among the rays of its bin (the count the
// atomic returns), so the scatter needs no atomics of its own.
__global__ void __launch_bounds__(256) k_sort_hist(const float4* __restrict__ rays, uint64_t n, KeyParams kp,
                                                   uint32_t* __restrict__ keys, uint32_t* __restrict__ ranks,
                                                   uint32_t* __restrict__ hist) {
    const uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const uint32_t key = ray_key(__ldg(rays + 2 * i), __ldg(rays + 2 * i + 1), kp);
    keys[i] = key;
    ranks[i] = atomicAdd(hist + key, 1u);
}

// Exclusive scan of the `nbins` counters in tiles of kScanTile: each block
// scans one tile in shared memory (loads and stores coalesced; a thread owns
// 8 consecutive counters) and records the tile's total; a second launch adds
// the totals of the earlier tiles.  nbins <= 2^18, so at most 32 tiles.
constexpr uint32_t kScanTile = 8192;
constexpr uint32_t kScanMaxTiles = 32;

__global__ void __launch_bounds__(1024) k_sort_scan_tiles(uint32_t* __restrict__ hist, uint32_t nbins,
                                                          uint32_t* __restrict__ tile_sums) {
    __shared__ uint32_t s[kScanTile];
    __shared__ uint32_t warp_excl[32];
    const uint32_t t = threadIdx.x, lane = t & 31u, warp = t >> 5;
    const uint32_t base = blockIdx.x * kScanTile;
    for (uint32_t k = t; k < kScanTile; k += 1024) s[k] = base + k < nbins ? hist[base + k] : 0u;
    __syncthreads();
    uint32_t v[8], sum = 0;
#pragma unroll
    for (int k = 0; k < 8; k++) {
        v[k] = s[t * 8 + k];
        sum += v[k];
    }
    uint32_t incl = sum;  // inclusive scan of the threads' sums within the warp
#pragma unroll
    for (uint32_t o = 1; o < 32; o <<= 1) {
        const uint32_t y = __shfl_up_sync(0xffffffffu, incl, o);
        if (lane >= o) incl += y;
    }
    if (lane == 31) warp_excl[warp] = incl;
    __syncthreads();
    if (warp == 0) {
        const uint32_t w = warp_excl[lane];
        uint32_t wi = w;
#pragma unroll
        for (uint32_t o = 1; o < 32; o <<= 1) {
            const uint32_t y = __shfl_up_sync(0xffffffffu, wi, o);
            if (lane >= o) wi += y;
        }
        warp_excl[lane] = wi - w;
        if (lane == 31) tile_sums[blockIdx.x] = wi;
    }
    __syncthreads();
    uint32_t run = warp_excl[warp] + incl - sum;  // counters before this thread's 8 in the tile
#pragma unroll
    for (int k = 0; k < 8; k++) {
        s[t * 8 + k] = run;
        run += v[k];
    }
    __syncthreads();
    for (uint32_t k = t; k < kScanTile; k += 1024)
        if (base + k < nbins) hist[base + k] = s[k];
}

__global__ void __launch_bounds__(1024) k_sort_scan_add(uint32_t* __restrict__ hist, uint32_t nbins,
                                                        const uint32_t* __restrict__ tile_sums) {
    __shared__ uint32_t off;
    if (threadIdx.x < 32) {
        uint32_t x = threadIdx.x < blockIdx.x ? tile_sums[threadIdx.x] : 0u;
#pragma unroll
        for (uint32_t o = 16; o > 0; o >>= 1) x += __shfl_xor_sync(0xffffffffu, x, o);
        if (threadIdx.x == 0) off = x;
    }
    __syncthreads();
    const uint32_t base = blockIdx.x * kScanTile;
    for (uint32_t k = threadIdx.x; k < kScanTile; k += 1024)
        if (base + k < nbins) hist[base + k] += off;
}

// Ray i goes to position pos = offset(key) + rank: its copy is written
// there, and pos replaces its rank (the gather of the hits reads it).
__global__ void __launch_bounds__(256) k_sort_scatter(const uint32_t* __restrict__ keys,
                                                      uint32_t* __restrict__ ranks, uint64_t n,
                                                      const uint32_t* __restrict__ offsets,
                                                      const float4* __restrict__ rays,
                                                      float4* __restrict__ sorted) {
    const uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const uint32_t pos = __ldg(offsets + keys[i]) + ranks[i];
    ranks[i] = pos;
    if (pos < n) {  // always true when the offsets are right
        const float4 a = __ldcs(rays + 2 * i), b = __ldcs(rays + 2 * i + 1);
        sorted[2 * (uint64_t)pos] = a;
        sorted[2 * (uint64_t)pos + 1] = b;
    }
}

// Hit i of the caller's order = sorted hit pos[i].
template <class T>
__global__ void __launch_bounds__(256) k_unsort_hits(const T* __restrict__ sorted, const uint32_t* __restrict__ pos,
                                                     uint64_t n, T* __restrict__ hits) {
    const uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const uint32_t p = __ldg(pos + i);
    if (p < n) __stcs(hits + i, __ldg(sorted + p));
}

}  // namespace

// Device scratch of a sorted trace of n rays: the sorted rays (32 B each)
// and hits (hit_bytes each), then keys and ranks/positions (4 B each), the
// bins and the scan's tile totals.
uint64_t sort_scratch_bytes(const int ldim[3], int g, uint64_t n, uint32_t hit_bytes, uint32_t* nbins_out) {
    int mbits = 0;
    for (int i = 0; i < 3; i++) {
        int b = ldim[i] - g;
        if (b < 0) b = 0;
        if (b > 5) b = 5;  // at most 2^18 bins in all
        mbits += b;
    }
    const uint32_t nbins = 8u << mbits;
    if (nbins_out) *nbins_out = nbins;
    return n * (32ull + hit_bytes + 8ull) + ((uint64_t)nbins + kScanMaxTiles) * sizeof(uint32_t) + 256;
}

// Sorts the rays into scratch: *sorted_rays receives the rays in key order,
// *sorted_hits the space for their hits, *pos each ray's position in it.
int sort_rays(const int ldim[3], int g, const vx_ray* rays, uint64_t n, uint32_t hit_bytes, void* scratch,
              SortedRays* out, cudaStream_t st) {
    if (n >= 0xFFFFFFFFull) return fail(VX_EINVAL, "sorted tracing supports fewer than 2^32 rays per call");
    KeyParams kp;
    kp.g = g;
    kp.mbits = 0;
    for (int i = 0; i < 3; i++) {
        kp.ld[i] = ldim[i];
        int b = ldim[i] - g;
        if (b < 0) b = 0;
        if (b > 5) b = 5;
        kp.kb[i] = b;
        kp.sh[i] = ldim[i] - b;
        kp.mbits += b;
    }
    const uint32_t nbins = 8u << kp.mbits;
    char* base = static_cast<char*>(scratch);
    float4* sorted = reinterpret_cast<float4*>(base);
    void* shits = base + 32 * n;
    uint32_t* keys = reinterpret_cast<uint32_t*>(base + (32ull + hit_bytes) * n);
    uint32_t* ranks = keys + n;
    uint32_t* hist = ranks + n;
    uint32_t* tile_sums = hist + nbins;
    const uint32_t tiles = (nbins + kScanTile - 1) / kScanTile;
    cudaError_t e = cudaMemsetAsync(hist, 0, (size_t)nbins * sizeof(uint32_t), st);
    if (e) return fail(VX_ECUDA, "sort memset: %s", cudaGetErrorString(e));
    const unsigned grid = (unsigned)((n + 255) / 256);
    const float4* r4 = reinterpret_cast<const float4*>(rays);
    k_sort_hist<<<grid, 256, 0, st>>>(r4, n, kp, keys, ranks, hist);
    k_sort_scan_tiles<<<tiles, 1024, 0, st>>>(hist, nbins, tile_sums);
    if (tiles > 1) k_sort_scan_add<<<tiles, 1024, 0, st>>>(hist, nbins, tile_sums);
    k_sort_scatter<<<grid, 256, 0, st>>>(keys, ranks, n, hist, r4, sorted);
    e = cudaGetLastError();
    if (e) return fail(VX_ECUDA, "sort launch: %s", cudaGetErrorString(e));
    out->rays = reinterpret_cast<const vx_ray*>(sorted);
    out->hits = shits;
    out->pos = ranks;
    return VX_OK;
}

// Puts the hits of a sorted trace back in the caller's order.
int unsort_hits(const SortedRays& s, uint64_t n, void* hits, int layout, cudaStream_t st) {
    if (n == 0) return VX_OK;
    const unsigned grid = (unsigned)((n + 255) / 256);
    if (layout == VX_HIT_FULL)
        k_unsort_hits<uint4><<<grid, 256, 0, st>>>(static_cast<const uint4*>(s.hits), s.pos, n,
                                                   static_cast<uint4*>(hits));
    else
        k_unsort_hits<uint2><<<grid, 256, 0, st>>>(static_cast<const uint2*>(s.hits), s.pos, n,
                                                   static_cast<uint2*>(hits));
    cudaError_t e = cudaGetLastError();
    if (e) return fail(VX_ECUDA, "unsort launch: %s", cudaGetErrorString(e));
    return VX_OK;
}

}  // namespace vx
