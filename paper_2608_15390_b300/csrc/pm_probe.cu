// pm_probe.cu -- on-chip bandwidth probes: the denominators of the roofline
// of a path whose state and matrices stay in shared memory and L2.
//
//   l2_read_probe    streaming 16-byte reads (ld.global.cg: cached in L2,
//                    not in L1) of a buffer smaller than L2, repeated, so
//                    after the first pass every read is an L2 hit;
//   smem_read_probe  16-byte reads of a block's shared memory, consecutive
//                    lanes on consecutive words (no bank conflicts).
// Both fold what they read into a value that is written only if it matches
// an unlikely constant, so the loads are not removed.
#include <cstdint>
#include <cuda_runtime.h>

#include "pm_internal.h"

namespace pm {

namespace {

__global__ void __launch_bounds__(512) l2_read_probe(const uint4* __restrict__ buf, size_t n16, int iters,
                                                     unsigned long long* sink)
{
    uint32_t acc = 0;
    const size_t stride = (size_t)gridDim.x * blockDim.x;
    for (int it = 0; it < iters; ++it) {
        for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < n16; i += 4 * stride) {
            uint4 v[4];
#pragma unroll
            for (int u = 0; u < 4; ++u) v[u] = (i + u * stride < n16) ? __ldcg(buf + i + u * stride) : make_uint4(0, 0, 0, 0);
#pragma unroll
            for (int u = 0; u < 4; ++u) acc ^= v[u].x ^ v[u].y ^ v[u].z ^ v[u].w;
        }
    }
    if (acc == 0x9E3779B9u) atomicAdd(sink, 1ull);
}

__global__ void __launch_bounds__(512) smem_read_probe(int words16, int iters, unsigned long long* sink)
{
    extern __shared__ uint4 sm[];
    for (int i = threadIdx.x; i < words16; i += blockDim.x)
        sm[i] = make_uint4(i, i * 3u, i * 5u, i * 7u + blockIdx.x);
    __syncthreads();
    uint32_t acc = 0;
    for (int it = 0; it < iters; ++it) {
        const int base = (it * 32) % words16;
#pragma unroll 4
        for (int i = threadIdx.x; i < words16; i += blockDim.x) {
            int j = i + base;
            j = j >= words16 ? j - words16 : j;
            const uint4 v = sm[j];
            acc ^= v.x ^ v.y ^ v.z ^ v.w;
        }
    }
    if (acc == 0x9E3779B9u) atomicAdd(sink, 1ull);
}

}  // namespace

cudaError_t launch_l2_probe(const void* buf, size_t bytes, int iters, int grid, unsigned long long* sink,
                            cudaStream_t st)
{
    l2_read_probe<<<grid, 512, 0, st>>>(reinterpret_cast<const uint4*>(buf), bytes / 16, iters, sink);
    return cudaGetLastError();
}

cudaError_t launch_smem_probe(int smem_bytes, int iters, int grid, unsigned long long* sink, cudaStream_t st)
{
    cudaError_t e = cudaFuncSetAttribute(smem_read_probe, cudaFuncAttributeMaxDynamicSharedMemorySize, smem_bytes);
    if (e != cudaSuccess) return e;
    smem_read_probe<<<grid, 512, smem_bytes, st>>>(smem_bytes / 16, iters, sink);
    return cudaGetLastError();
}

}  // namespace pm
