// pm_noalloc.cu -- statistics of a device array of log-weights without any
// allocation, for callers that cannot allocate device memory when they call
// in: hosts whose own allocator has reserved the device memory and leaves
// none for a library, and loops that cannot afford the device-wide
// synchronisation cudaMalloc / cudaFree may cause.
//
// The reduction runs the same two kernels as the statistics step of
// estimate_permanent; their per-chunk partial sums live in one file-scope
// device array that every GPU loading this library holds until the process
// exits (kNoAllocScratchBytes, about 50 KB).
#include <cstdint>
#include <mutex>

#include "../../include/pm.h"
#include "pm_internal.h"

namespace {

constexpr uint64_t kNoAllocChunkLen = 65536;   // log-weights per partial sum
constexpr int kNoAllocMaxChunks = 1024;        // partial sums the scratch holds
constexpr uint64_t kNoAllocMaxM = kNoAllocChunkLen * kNoAllocMaxChunks;  // 2^26
constexpr size_t kNoAllocPrefixOff = 0;        // two uint64: {0, M}
constexpr size_t kNoAllocPartOff = 256;
constexpr size_t kNoAllocScratchBytes = kNoAllocPartOff + sizeof(pm::StatsPartial) * kNoAllocMaxChunks;

static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocScratchBytes];

static_assert(sizeof(pm_weight_stats) == sizeof(pm::StatsOut), "pm_weight_stats must mirror StatsOut");

constexpr int kMaxDevices = 64;
std::mutex g_setup_mutex;
void* g_scratch_addr[kMaxDevices] = {};

// the device address of the scratch array on the current device (host code
// only sees a stand-in symbol, so the address is looked up once per device)
cudaError_t scratch_address(int dev, void** out)
{
    std::lock_guard<std::mutex> lock(g_setup_mutex);
    if (!g_scratch_addr[dev]) {
        void* p = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess) return e;
        g_scratch_addr[dev] = p;
    }
    *out = g_scratch_addr[dev];
    return cudaSuccess;
}

__global__ void noalloc_prefix_kernel(uint64_t* prefix, uint64_t M)
{
    prefix[0] = 0;
    prefix[1] = M;
}

}  // namespace

extern "C" pm_status pm_log_weight_stats_noalloc(const double* log_x, uint64_t M, pm_weight_stats* out,
                                                 void* cuda_stream)
{
    if (!log_x || !out || M == 0) return PM_EINVAL;
    if (M > kNoAllocMaxM) return PM_EUNSUPPORTED;  // more log-weights than the fixed scratch can reduce
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return PM_ECUDA;
    if (dev < 0 || dev >= kMaxDevices) return PM_EUNSUPPORTED;
    void* base = nullptr;
    if (scratch_address(dev, &base) != cudaSuccess) return PM_ECUDA;
    cudaStream_t st = (cudaStream_t)cuda_stream;
    uint64_t* prefix = reinterpret_cast<uint64_t*>(static_cast<unsigned char*>(base) + kNoAllocPrefixOff);
    pm::StatsPartial* parts =
        reinterpret_cast<pm::StatsPartial*>(static_cast<unsigned char*>(base) + kNoAllocPartOff);
    const int chunks = (int)((M + kNoAllocChunkLen - 1) / kNoAllocChunkLen);
    // every partial read by the merge is rewritten first, so nothing in the
    // scratch has to start at zero
    noalloc_prefix_kernel<<<1, 1, 0, st>>>(prefix, M);
    if (cudaGetLastError() != cudaSuccess) return PM_ECUDA;
    if (pm::launch_stats(log_x, nullptr, prefix, 1, parts, chunks, reinterpret_cast<pm::StatsOut*>(out), st) !=
        cudaSuccess)
        return PM_ECUDA;
    return PM_OK;
}
