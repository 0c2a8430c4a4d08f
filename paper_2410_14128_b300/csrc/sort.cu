// sort.cu -- ray sorting for coherence before tracing.
//
// Key of a ray = direction octant (3 bits) above the Morton code (x lowest,
// Fig. 5 order) of its origin's cell of side 2^g voxels, the origin clamped
// into the grid.  Rays with equal keys start close together and head the
// same way, so a warp that traces consecutive sorted rays reads the same
// nodes and takes similar paths.  A counting sort by key (histogram,
// exclusive scan, scatter) yields `order`, the ray indices in key order; the
// trace kernels read rays and write hits through it, so results stay in the
// caller's order.
#include <cuda_runtime.h>

#include "trace.cuh"
#include "vx_internal.hpp"

namespace vx {
namespace {

struct KeyParams {
    int ld[3];
    int g;      // cell side 2^g
    int kb[3];  // Morton bits per axis
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
        cell[i] = ((uint32_t)v) >> k.g;
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

__global__ void __launch_bounds__(256) k_sort_hist(const float4* __restrict__ rays, uint64_t n, KeyParams kp,
                                                   uint32_t* __restrict__ keys, uint32_t* __restrict__ hist) {
    const uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const uint32_t key = ray_key(__ldg(rays + 2 * i), __ldg(rays + 2 * i + 1), kp);
    keys[i] = key;
    atomicAdd(hist + key, 1u);
}

// In-place exclusive scan of `nbins` counters with one block of 1024 threads.
__global__ void __launch_bounds__(1024) k_sort_scan(uint32_t* __restrict__ hist, uint32_t nbins) {
    __shared__ uint32_t part[1024];
    const uint32_t t = threadIdx.x;
    const uint32_t per = (nbins + 1023) / 1024;
    const uint32_t lo = t * per, hi = min(lo + per, nbins);
    uint32_t sum = 0;
    for (uint32_t i = lo; i < hi; i++) sum += hist[i];
    part[t] = sum;
    __syncthreads();
    for (uint32_t off = 1; off < 1024; off <<= 1) {
        const uint32_t v = t >= off ? part[t - off] : 0u;
        __syncthreads();
        part[t] += v;
        __syncthreads();
    }
    uint32_t run = part[t] - sum;  // exclusive prefix of this thread's chunk
    for (uint32_t i = lo; i < hi; i++) {
        const uint32_t c = hist[i];
        hist[i] = run;
        run += c;
    }
}

__global__ void __launch_bounds__(256) k_sort_scatter(const uint32_t* __restrict__ keys, uint64_t n,
                                                      uint32_t* __restrict__ offsets, uint32_t* __restrict__ order) {
    const uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const uint32_t pos = atomicAdd(offsets + keys[i], 1u);
    order[pos] = (uint32_t)i;
}

}  // namespace

// Bytes of device scratch sort_rays needs for n rays.
uint64_t sort_scratch_bytes(const int ldim[3], int g, uint64_t n, uint32_t* nbins_out) {
    int mbits = 0;
    for (int i = 0; i < 3; i++) {
        int b = ldim[i] - g;
        if (b < 0) b = 0;
        if (b > 5) b = 5;  // at most 2^18 bins in all
        mbits += b;
    }
    const uint32_t nbins = 8u << mbits;
    if (nbins_out) *nbins_out = nbins;
    return 2 * n * sizeof(uint32_t) + (uint64_t)nbins * sizeof(uint32_t) + 256;
}

// Fills order[0..n) (inside `scratch`) with ray indices sorted by key.
int sort_rays(const int ldim[3], int g, const vx_ray* rays, uint64_t n, void* scratch, uint32_t** order_out,
              cudaStream_t st) {
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
        kp.mbits += b;
    }
    const uint32_t nbins = 8u << kp.mbits;
    uint32_t* keys = static_cast<uint32_t*>(scratch);
    uint32_t* order = keys + n;
    uint32_t* hist = order + n;
    cudaError_t e = cudaMemsetAsync(hist, 0, (size_t)nbins * sizeof(uint32_t), st);
    if (e) return fail(VX_ECUDA, "sort memset: %s", cudaGetErrorString(e));
    const unsigned grid = (unsigned)((n + 255) / 256);
    k_sort_hist<<<grid, 256, 0, st>>>(reinterpret_cast<const float4*>(rays), n, kp, keys, hist);
    k_sort_scan<<<1, 1024, 0, st>>>(hist, nbins);
    k_sort_scatter<<<grid, 256, 0, st>>>(keys, n, hist, order);
    e = cudaGetLastError();
    if (e) return fail(VX_ECUDA, "sort launch: %s", cudaGetErrorString(e));
    *order_out = order;
    return VX_OK;
}

}  // namespace vx
