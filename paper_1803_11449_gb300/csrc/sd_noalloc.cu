// sd_noalloc.cu -- sd_update_noalloc: the binned DHLA update (Algorithm 1,
// the k_bin / k_apply kernels of sd_binned.cu) for callers that must not
// allocate device memory.
//
// Who needs it: a packet-ingest thread on a latency budget (cudaMalloc can
// synchronise the whole device and take milliseconds), and programs whose
// device memory is entirely owned by another allocator (a framework's
// caching allocator, or a pool reserved at start-up) where an extra
// cudaMalloc may fail or fragment the pool.  The caller passes the pairs and
// the DHLA it owns; the entry point allocates nothing.
//
// Its scratch (the bins, their counters and the apply work counter) is the
// file-scope array below.  Every GPU that loads this library holds the array
// until the process exits.  All calls share it and it keeps the last call's
// contents, so each call clears the counters it relies on; calls whose work
// overlaps on the GPU (different streams, or different host threads) race on
// it and must be serialised by the caller.
//
// Launch failures are read from the runtime's per-thread error state, which
// also holds errors that earlier, unrelated runtime calls left there.  So a
// call first looks at that state without clearing it, and when an error is
// already pending it returns SD_ERR_CUDA with nothing queued: it neither
// reports nor consumes the caller's own error.
#include <cstring>
#include <mutex>

#include "sd.h"
#include "sd_common.cuh"

namespace {

// 16 MiB of 32-bit words: bins for 4096 slices at most, plus counters.
constexpr uint64_t kScratchWords = 4ull << 20;
static __device__ __align__(256) uint32_t g_noalloc_scratch[kScratchWords];

// Device address of g_noalloc_scratch per device, looked up once per device.
constexpr int kMaxDevices = 64;
std::mutex g_mu;
uint32_t *g_addr[kMaxDevices] = {nullptr};

__global__ void k_clear_counts(uint32_t *p, uint32_t n) {
    for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) p[i] = 0;
}

}  // namespace

extern "C" int sd_update_noalloc(const sd_params *p, uint32_t *grid, const uint32_t *pairs, uint64_t n,
                                 void *cuda_stream) {
    using namespace sd;
    if (sd_check_params(p) != SD_OK || !grid || (n && !pairs) || ((uintptr_t)pairs & 3u) ||
        ((uintptr_t)grid & 15u))
        return SD_ERR_ARG;
    if (n == 0) return SD_OK;
    if (cudaPeekAtLastError() != cudaSuccess) return SD_ERR_CUDA;  // an earlier call's error is pending
    int dev = -1;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) return SD_ERR_CUDA;
    // both buffers must be device (or managed) memory of the current device
    for (const void *ptr : {static_cast<const void *>(grid), static_cast<const void *>(pairs)}) {
        cudaPointerAttributes a;
        if (cudaPointerGetAttributes(&a, ptr) != cudaSuccess) {
            cudaGetLastError();  // the lookup's own error (none was pending before it)
            return SD_ERR_ARG;
        }
        if (a.type == cudaMemoryTypeDevice && a.device != dev) return SD_ERR_ARG;
        if (a.type != cudaMemoryTypeDevice && a.type != cudaMemoryTypeManaged) return SD_ERR_ARG;
    }

    // set-up, once per device, with that device current
    uint32_t *scratch = nullptr;
    {
        std::lock_guard<std::mutex> lock(g_mu);
        if (!g_addr[dev]) {
            void *a = nullptr;
            if (cudaGetSymbolAddress(&a, g_noalloc_scratch) != cudaSuccess || !a) return SD_ERR_CUDA;
            g_addr[dev] = static_cast<uint32_t *>(a);
        }
        scratch = g_addr[dev];
    }

    // geometry and hash constants, as for a handle with the same parameters
    Geometry G;
    geometry_of(p, &G);

    // slices of 2^15 words (at most 4096: a DHLA of up to 512 MiB); bins sized
    // to the scratch, rounds sized to the bins with 100% slack for skew
    const uint64_t total = (uint64_t)G.dirs * G.dir_words;
    uint32_t sl = 15;
    while (sl > 10 && (1ull << (sl - 1)) >= total) sl--;
    const uint64_t S = (total + (1ull << sl) - 1) >> sl;
    if (S > 4096) return SD_ERR_TOO_LARGE;  // more than 512 MiB of DHLA
    const uint64_t cap = ((kScratchWords - S - 4) / S) & ~3ull;
    const uint64_t per_pair = (uint64_t)G.dirs * G.r;
    const uint64_t chunk = cap * S / (2 * per_pair);
    if (cap < 256 || chunk < 1024) return SD_ERR_TOO_LARGE;  // bins would not fit the scratch

    BinArgs B;
    std::memset(&B, 0, sizeof B);
    B.bins = scratch;
    B.count = scratch + S * cap;
    B.work = B.count + S;
    B.S = (uint32_t)S;
    B.slice_log2 = sl;
    B.cap = (uint32_t)cap;
    B.tile_pairs = per_pair > 8 ? 512 : 1024;  // shared memory of one binning tile
    B.total_words = total;
    if (bin_smem_bytes(B.tile_pairs, (uint32_t)per_pair, B.S) > 200 * 1024) return SD_ERR_TOO_LARGE;

    int num_sms = 0;
    if (cudaDeviceGetAttribute(&num_sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return SD_ERR_CUDA;
    cudaStream_t s = (cudaStream_t)cuda_stream;
    // the counters start at zero; the array keeps whatever the last call left
    uint32_t *counts = B.count;
    uint32_t ncount = (uint32_t)(S + 4);
    void *args[] = {&counts, &ncount};
    if (cudaLaunchKernel(reinterpret_cast<const void *>(k_clear_counts), dim3(1), dim3(256), args, 0, s) !=
        cudaSuccess) {
        cudaGetLastError();
        return SD_ERR_CUDA;
    }
    for (uint64_t off = 0; off < n; off += chunk) {
        const uint64_t m = n - off < chunk ? n - off : chunk;
        if (launch_binned_chunk(pairs + 2 * off, m, grid, G, B, num_sms, s) != cudaSuccess) return SD_ERR_CUDA;
    }
    return SD_OK;
}
