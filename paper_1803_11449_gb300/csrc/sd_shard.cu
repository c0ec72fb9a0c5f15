// sd_shard.cu -- device steps of running one detection over several GPUs.
//
// Two ways to spread a window over GPUs, both from the paper:
//
//   * stream split, then merge (§4.2: local DHLAs merged into a global one,
//     read as a bitwise OR): every GPU runs Algorithm 1 on its part of the
//     stream; the DHLA images are then ORed across GPUs.  The collective
//     (reduce-scatter by all-to-all, all-gather) is issued by the caller;
//     the OR of the gathered parts is k_or_words here.
//   * key partition (§5: hosts divided by the low bits of their address):
//     the pairs of each direction are grouped by key & (parts - 1) and sent
//     to the GPU that owns those keys; each GPU keeps a DHLA of its own keys
//     and nothing is merged.  The grouping is k_part_count / k_part_scatter:
//     a counting pass, then a scatter of (key, peer) pairs into one segment
//     per part, each block reserving its runs with one atomic per part.
#include "sd_common.cuh"

namespace sd {

namespace {

constexpr uint32_t kMaxParts = 1024;

}  // namespace

// dst[j] = src[0 * words + j] | src[1 * words + j] | ... | src[(count-1) * words + j]
__global__ void k_or_words(uint4 *__restrict__ dst, const uint4 *__restrict__ src, uint64_t words4, uint32_t count) {
    const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
    for (uint64_t j = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; j < words4; j += stride) {
        uint4 a = __ldg(src + j);
        for (uint32_t i = 1; i < count; i++) {
            const uint4 b = __ldg(src + (uint64_t)i * words4 + j);
            a.x |= b.x; a.y |= b.y; a.z |= b.z; a.w |= b.w;
        }
        dst[j] = a;
    }
}

__device__ __forceinline__ uint32_t part_key(const uint32_t *pairs, uint64_t p, uint32_t dir) {
    return ld_stream_u32(pairs + 2 * p + (dir ? 1 : 0));
}

// counts[q] += pairs whose key (src for dir 0, dst for dir 1) has
// key & (parts - 1) == q
__global__ void __launch_bounds__(256)
k_part_count(const uint32_t *__restrict__ pairs, uint64_t n, uint32_t dir, uint32_t parts,
             unsigned long long *__restrict__ counts) {
    __shared__ uint32_t hist[kMaxParts];
    for (uint32_t q = threadIdx.x; q < parts; q += blockDim.x) hist[q] = 0;
    __syncthreads();
    const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
    for (uint64_t p = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; p < n; p += stride)
        atomicAdd(&hist[part_key(pairs, p, dir) & (parts - 1)], 1u);
    __syncthreads();
    for (uint32_t q = threadIdx.x; q < parts; q += blockDim.x)
        if (hist[q]) atomicAdd(&counts[q], (unsigned long long)hist[q]);
}

// Each block takes a contiguous range of pairs, counts its pairs per part,
// reserves one run per part behind cursor[q] (which starts at part q's
// offset), and writes its (key, peer) pairs there.
__global__ void __launch_bounds__(256)
k_part_scatter(const uint32_t *__restrict__ pairs, uint64_t n, uint32_t dir, uint32_t parts,
               unsigned long long *__restrict__ cursor, uint32_t *__restrict__ out) {
    __shared__ uint32_t hist[kMaxParts];
    __shared__ unsigned long long base[kMaxParts];
    const uint64_t per = (n + gridDim.x - 1) / gridDim.x;
    const uint64_t p0 = (uint64_t)blockIdx.x * per;
    const uint64_t p1 = p0 + per < n ? p0 + per : n;
    for (uint32_t q = threadIdx.x; q < parts; q += blockDim.x) hist[q] = 0;
    __syncthreads();
    for (uint64_t p = p0 + threadIdx.x; p < p1; p += blockDim.x)
        atomicAdd(&hist[part_key(pairs, p, dir) & (parts - 1)], 1u);
    __syncthreads();
    for (uint32_t q = threadIdx.x; q < parts; q += blockDim.x) {
        base[q] = hist[q] ? atomicAdd(&cursor[q], (unsigned long long)hist[q]) : 0ull;
        hist[q] = 0;
    }
    __syncthreads();
    for (uint64_t p = p0 + threadIdx.x; p < p1; p += blockDim.x) {
        const uint32_t s = ld_stream_u32(pairs + 2 * p), t = ld_stream_u32(pairs + 2 * p + 1);
        const uint32_t key = dir ? t : s, peer = dir ? s : t;
        const uint32_t q = key & (parts - 1);
        const unsigned long long at = base[q] + atomicAdd(&hist[q], 1u);
        out[2 * at] = key;
        out[2 * at + 1] = peer;
    }
}

cudaError_t launch_or_words(uint32_t *dst, const uint32_t *src, uint64_t words, uint32_t count, int num_sms,
                            cudaStream_t s) {
    const uint64_t w4 = words / 4;
    uint64_t blocks = (w4 + 255) / 256;
    if (blocks > (uint64_t)num_sms * 8) blocks = (uint64_t)num_sms * 8;
    if (blocks == 0) blocks = 1;
    k_or_words<<<(unsigned)blocks, 256, 0, s>>>(reinterpret_cast<uint4 *>(dst), reinterpret_cast<const uint4 *>(src),
                                                 w4, count);
    return cudaGetLastError();
}

cudaError_t launch_partition(const uint32_t *pairs, uint64_t n, uint32_t dir, uint32_t parts,
                             unsigned long long *counts, unsigned long long *cursor, uint32_t *out, int num_sms,
                             cudaStream_t s, bool scatter) {
    uint64_t blocks = (n + 255) / 256;
    if (blocks > (uint64_t)num_sms * 8) blocks = (uint64_t)num_sms * 8;
    if (blocks == 0) blocks = 1;
    if (!scatter) {
        k_part_count<<<(unsigned)blocks, 256, 0, s>>>(pairs, n, dir, parts, counts);
    } else {
        k_part_scatter<<<(unsigned)blocks, 256, 0, s>>>(pairs, n, dir, parts, cursor, out);
    }
    return cudaGetLastError();
}

}  // namespace sd
