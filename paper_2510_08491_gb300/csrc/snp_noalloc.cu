// snp_noalloc.cu -- an allocation-free entry point: the stable radix sort of
// (u64 key, u32 value) pairs that orders the tile keys, with all of its scratch
// (ping-pong key/value buffers, digit histograms, scan partials, the device copy
// of the item count) in one file-scope device array instead of context
// workspace.
//
// Who needs it: callers that must not allocate device memory while they run --
// renderers embedded in an application whose memory pool owns the whole device
// (a cudaMalloc there fails or steals the pool's memory), plugins that are handed
// a fixed arena and nothing else, or real-time loops that cannot afford the
// implicit device synchronisation of cudaMalloc / cudaFree.  They pass their own
// key and value arrays; nothing else is needed.
//
// The array is SNP_NOALLOC_SORT_BYTES large and lives on every device that loads
// the library until the process exits.  All calls share it and it keeps what the
// last call left there; every call overwrites the parts it reads before reading
// them, so nothing has to start at zero.  Two calls whose work overlaps on the GPU
// (different streams, or different host threads on one device) race on the array.
#include <cuda_runtime.h>
#include <stdint.h>

#include <mutex>

#include "snp.h"
#include "snp_common.cuh"
#include "snp_internal.h"

namespace snp {
namespace {

constexpr int64_t kNoallocMax = SNP_NOALLOC_SORT_MAX;
constexpr int64_t kBlockItems = 4096;  // items per radix block (matches the sort kernels)
constexpr int64_t kHistWords = 256 * (kNoallocMax / kBlockItems);
constexpr int64_t kScanWords = 256;  // >= scan_temp_words(kHistWords), checked at set-up

// Byte offsets inside the scratch array.
constexpr size_t kOffKeys = 0;
constexpr size_t kOffVals = kOffKeys + (size_t)kNoallocMax * 8;
constexpr size_t kOffHist = kOffVals + (size_t)kNoallocMax * 4;
constexpr size_t kOffHistScan = kOffHist + (size_t)kHistWords * 4;
constexpr size_t kOffScan = kOffHistScan + (size_t)kHistWords * 4;
constexpr size_t kOffN = kOffScan + (size_t)kScanWords * 4;
constexpr size_t kBytes = kOffN + 256;
static_assert(kBytes <= SNP_NOALLOC_SORT_BYTES, "scratch layout exceeds SNP_NOALLOC_SORT_BYTES");

}  // namespace

__device__ __align__(256) unsigned char g_noalloc_scratch[SNP_NOALLOC_SORT_BYTES];

__global__ void k_noalloc_set_count(uint32_t *dst, uint32_t n) { *dst = n; }

namespace {

constexpr int kMaxDevices = 64;
std::mutex g_mu;
unsigned char *g_ptr[kMaxDevices] = {nullptr};

// Device address of the scratch array on the current device (looked up once per device).
snp_status scratch_on_current_device(unsigned char **out)
{
    int dev = -1;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) return SNP_ERR_CUDA;
    std::lock_guard<std::mutex> lk(g_mu);
    if (!g_ptr[dev]) {
        void *p = nullptr;
        if (cudaGetSymbolAddress(&p, g_noalloc_scratch) != cudaSuccess || p == nullptr) return SNP_ERR_CUDA;
        if (scan_temp_words(kHistWords) > kScanWords) return SNP_ERR_UNSUPPORTED;
        g_ptr[dev] = (unsigned char *)p;
    }
    *out = g_ptr[dev];
    return SNP_OK;
}

}  // namespace
}  // namespace snp

extern "C" snp_status snp_sort_pairs_noalloc(uint64_t *keys, uint32_t *vals, int64_t n, int32_t key_bits,
                                             void *stream)
{
    using namespace snp;
    if (n < 0 || key_bits < 1 || key_bits > 64) return SNP_ERR_INVALID_ARG;
    if (n > kNoallocMax) return SNP_ERR_CAPACITY;
    if (n > 0 && (!keys || !vals)) return SNP_ERR_INVALID_ARG;
    // element alignment: a misaligned pointer would fault on the device instead
    if (((uintptr_t)keys & 7u) != 0 || ((uintptr_t)vals & 3u) != 0) return SNP_ERR_INVALID_ARG;
    unsigned char *base = nullptr;
    snp_status s = scratch_on_current_device(&base);
    if (s != SNP_OK) return s;
    if (n <= 1) return SNP_OK;
    cudaStream_t st = (cudaStream_t)stream;
    uint32_t *d_n = (uint32_t *)(base + kOffN);
    k_noalloc_set_count<<<1, 1, 0, st>>>(d_n, (uint32_t)n);
    note_launch();
    uint64_t *keys_alt = (uint64_t *)(base + kOffKeys);
    uint32_t *vals_alt = (uint32_t *)(base + kOffVals);
    const bool in_alt = radix_sort(keys, vals, keys_alt, vals_alt, d_n, n, key_bits, (uint32_t *)(base + kOffHist),
                                   (uint32_t *)(base + kOffHistScan), (uint32_t *)(base + kOffScan), st);
    if (in_alt) {
        if (cudaMemcpyAsync(keys, keys_alt, (size_t)n * 8, cudaMemcpyDeviceToDevice, st) != cudaSuccess ||
            cudaMemcpyAsync(vals, vals_alt, (size_t)n * 4, cudaMemcpyDeviceToDevice, st) != cudaSuccess)
            return SNP_ERR_CUDA;
    }
    return cudaGetLastError() == cudaSuccess ? SNP_OK : SNP_ERR_CUDA;
}
