// sd_ceilings.cu -- microbenchmarks of the on-chip and host-link rates that
// bound the DHLA update, for the benchmark's roofline lines (built as its
// own small library, libsd_ceilings.so; not part of the detection API).
//
//   sdc_smem_or_rate   random 32-bit atomic ORs into a block's shared memory
//                      (the apply step of the binned updates sets every bit
//                      this way): atomics per second for the whole GPU.
//   sdc_l2_rates       sweeps of an L2-resident buffer: read, write, and the
//                      bulk OR reduction from shared memory
//                      (cp.reduce.async.bulk ... .or.b32) that merges bit
//                      planes into the plane-major DHLA copy.
//   sdc_host_link      host to device: cudaMemcpy from pinned memory, and
//                      kernel reads of mapped pinned and of pageable memory
//                      (the latter where the device reads pageable memory).
//
// Every kernel indexes within its buffers; nothing waits on another block.
#include <cstdint>
#include <cstdlib>
#include <cstring>

#include <cuda_runtime.h>

namespace {

__global__ void k_smem_or(uint32_t lw, uint32_t iters, uint32_t *out) {
    extern __shared__ uint32_t s[];
    const uint32_t words = 1u << lw;
    for (uint32_t i = threadIdx.x; i < words; i += blockDim.x) s[i] = 0;
    __syncthreads();
    uint32_t x = (blockIdx.x * 1024u + threadIdx.x) * 0x9E3779B9u + 12345u;
    for (uint32_t it = 0; it < iters; it++) {
        x = x * 1664525u + 1013904223u;  // an LCG per thread: random word and bit
        atomicOr(&s[x >> (32u - lw)], 1u << (x & 31u));
    }
    __syncthreads();
    uint32_t acc = 0;
    for (uint32_t i = threadIdx.x; i < words; i += blockDim.x) acc ^= s[i];
    if (acc == 0x12345678u) out[blockIdx.x] = acc;  // keeps the work observable
}

__global__ void k_read(const uint4 *__restrict__ p, uint64_t n4, uint32_t *out) {
    uint32_t acc = 0;
    for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n4; i += (uint64_t)gridDim.x * blockDim.x) {
        const uint4 v = p[i];
        acc ^= v.x ^ v.y ^ v.z ^ v.w;
    }
    if (acc == 0x12345678u) out[0] = acc;
}

__global__ void k_write(uint4 *p, uint64_t n4, uint32_t v) {
    for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n4; i += (uint64_t)gridDim.x * blockDim.x)
        p[i] = make_uint4(v, v, v, v);
}

// each block ORs its shared-memory region into regions of dst
__global__ void k_bulk_or(uint32_t *dst, uint64_t regions, uint32_t region_bytes) {
    extern __shared__ uint32_t s[];
    for (uint32_t i = threadIdx.x; i < region_bytes / 4; i += blockDim.x) s[i] = (i * 2654435761u) & 0x01010101u;
    __syncthreads();
    if (threadIdx.x == 0) {
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        for (uint64_t r = blockIdx.x; r < regions; r += gridDim.x) {
            uint32_t *d = dst + r * (region_bytes / 4);
            asm volatile("cp.reduce.async.bulk.global.shared::cta.bulk_group.or.b32 [%0], [%1], %2;"
                         ::"l"(d), "r"((uint32_t)__cvta_generic_to_shared(s)), "r"(region_bytes)
                         : "memory");
            asm volatile("cp.async.bulk.commit_group;" ::: "memory");
        }
        asm volatile("cp.async.bulk.wait_group 0;" ::: "memory");
    }
    __syncthreads();
}

float elapsed_ms(cudaEvent_t a, cudaEvent_t b) {
    float ms = 0.f;
    cudaEventElapsedTime(&ms, a, b);
    return ms;
}

struct Events {
    cudaEvent_t a = nullptr, b = nullptr;
    Events() {
        cudaEventCreate(&a);
        cudaEventCreate(&b);
    }
    ~Events() {
        cudaEventDestroy(a);
        cudaEventDestroy(b);
    }
};

}  // namespace

extern "C" {

// Atomic ORs per second into shared memory of 2^words_log2 words per block
// (words_log2 in 10..15), `threads` per block, `blocks_per_sm` per SM.
int sdc_smem_or_rate(uint32_t words_log2, uint32_t threads, uint32_t blocks_per_sm, double *ops_per_s) {
    if (!ops_per_s || words_log2 < 10 || words_log2 > 15 || threads < 32 || threads > 1024 || !blocks_per_sm)
        return -1;
    int dev = 0, nsm = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev))
        return -3;
    const size_t smem = (size_t)4 << words_log2;
    if (cudaFuncSetAttribute(k_smem_or, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess)
        return -3;
    uint32_t *out = nullptr;
    if (cudaMalloc(&out, (size_t)nsm * blocks_per_sm * 4) != cudaSuccess) return -2;
    const uint32_t blocks = (uint32_t)nsm * blocks_per_sm, iters = 4096;
    Events ev;
    k_smem_or<<<blocks, threads, smem>>>(words_log2, 64, out);
    cudaEventRecord(ev.a);
    k_smem_or<<<blocks, threads, smem>>>(words_log2, iters, out);
    cudaEventRecord(ev.b);
    const cudaError_t e = cudaEventSynchronize(ev.b);
    const double ms = elapsed_ms(ev.a, ev.b);
    cudaFree(out);
    if (e != cudaSuccess || cudaGetLastError() != cudaSuccess || ms <= 0) return -3;
    *ops_per_s = (double)blocks * threads * iters / (ms * 1e-3);
    return 0;
}

// GB/s of a read sweep, a write sweep and a bulk-OR sweep (from 32 KiB of
// shared memory per block) over a buffer of `bytes` (a multiple of 32 KiB),
// each the mean of 10 back-to-back sweeps after a warm one.
int sdc_l2_rates(uint64_t bytes, double *read_gbs, double *write_gbs, double *bulk_or_gbs) {
    const uint32_t region = 32768;
    if (!read_gbs || !write_gbs || !bulk_or_gbs || !bytes || bytes % region) return -1;
    int dev = 0, nsm = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev))
        return -3;
    uint4 *buf = nullptr;
    uint32_t *out = nullptr;
    if (cudaMalloc(&buf, bytes) != cudaSuccess) return -2;
    if (cudaMalloc(&out, 4) != cudaSuccess) {
        cudaFree(buf);
        return -2;
    }
    cudaMemset(buf, 1, bytes);
    const uint64_t n4 = bytes / 16;
    const uint32_t blocks = (uint32_t)nsm * 4;
    Events ev;
    k_read<<<blocks, 512>>>(buf, n4, out);
    cudaEventRecord(ev.a);
    for (int i = 0; i < 10; i++) k_read<<<blocks, 512>>>(buf, n4, out);
    cudaEventRecord(ev.b);
    cudaEventSynchronize(ev.b);
    *read_gbs = bytes / (elapsed_ms(ev.a, ev.b) / 10 * 1e-3) / 1e9;
    cudaEventRecord(ev.a);
    for (int i = 0; i < 10; i++) k_write<<<blocks, 512>>>(buf, n4, (uint32_t)i);
    cudaEventRecord(ev.b);
    cudaEventSynchronize(ev.b);
    *write_gbs = bytes / (elapsed_ms(ev.a, ev.b) / 10 * 1e-3) / 1e9;
    cudaFuncSetAttribute(k_bulk_or, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)region);
    k_bulk_or<<<(uint32_t)nsm * 2, 256, region>>>((uint32_t *)buf, bytes / region, region);
    cudaEventRecord(ev.a);
    for (int i = 0; i < 10; i++) k_bulk_or<<<(uint32_t)nsm * 2, 256, region>>>((uint32_t *)buf, bytes / region, region);
    cudaEventRecord(ev.b);
    const cudaError_t e = cudaEventSynchronize(ev.b);
    *bulk_or_gbs = bytes / (elapsed_ms(ev.a, ev.b) / 10 * 1e-3) / 1e9;
    cudaFree(buf);
    cudaFree(out);
    return (e == cudaSuccess && cudaGetLastError() == cudaSuccess) ? 0 : -3;
}

// Host-to-device GB/s over `bytes`: cudaMemcpy from pinned memory, a kernel
// reading mapped pinned memory, and a kernel reading pageable memory
// (0 when the device does not read pageable memory).
int sdc_host_link(uint64_t bytes, double *h2d_gbs, double *pinned_read_gbs, double *pageable_read_gbs) {
    if (!h2d_gbs || !pinned_read_gbs || !pageable_read_gbs || !bytes || bytes % 16) return -1;
    int dev = 0, nsm = 0, pageable = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev) ||
        cudaDeviceGetAttribute(&pageable, cudaDevAttrPageableMemoryAccess, dev))
        return -3;
    void *pin = nullptr, *d = nullptr, *dp = nullptr;
    uint32_t *out = nullptr;
    if (cudaHostAlloc(&pin, bytes, cudaHostAllocMapped) != cudaSuccess) return -2;
    if (cudaMalloc(&d, bytes) != cudaSuccess || cudaMalloc(&out, 4) != cudaSuccess) {
        cudaFreeHost(pin);
        cudaFree(d);
        return -2;
    }
    std::memset(pin, 1, bytes);
    cudaHostGetDevicePointer(&dp, pin, 0);
    Events ev;
    cudaMemcpy(d, pin, bytes, cudaMemcpyHostToDevice);
    cudaEventRecord(ev.a);
    for (int i = 0; i < 3; i++) cudaMemcpyAsync(d, pin, bytes, cudaMemcpyHostToDevice);
    cudaEventRecord(ev.b);
    cudaEventSynchronize(ev.b);
    *h2d_gbs = bytes / (elapsed_ms(ev.a, ev.b) / 3 * 1e-3) / 1e9;
    const uint64_t n4 = bytes / 16;
    k_read<<<(uint32_t)nsm * 4, 512>>>((const uint4 *)dp, n4, out);
    cudaEventRecord(ev.a);
    for (int i = 0; i < 3; i++) k_read<<<(uint32_t)nsm * 4, 512>>>((const uint4 *)dp, n4, out);
    cudaEventRecord(ev.b);
    cudaEventSynchronize(ev.b);
    *pinned_read_gbs = bytes / (elapsed_ms(ev.a, ev.b) / 3 * 1e-3) / 1e9;
    *pageable_read_gbs = 0.0;
    if (pageable) {
        void *pg = std::malloc(bytes);
        if (pg) {
            std::memset(pg, 1, bytes);
            k_read<<<(uint32_t)nsm * 4, 512>>>((const uint4 *)pg, n4, out);
            cudaDeviceSynchronize();
            cudaEventRecord(ev.a);
            for (int i = 0; i < 3; i++) k_read<<<(uint32_t)nsm * 4, 512>>>((const uint4 *)pg, n4, out);
            cudaEventRecord(ev.b);
            cudaEventSynchronize(ev.b);
            *pageable_read_gbs = bytes / (elapsed_ms(ev.a, ev.b) / 3 * 1e-3) / 1e9;
            std::free(pg);
        }
    }
    const cudaError_t e = cudaDeviceSynchronize();
    cudaFreeHost(pin);
    cudaFree(d);
    cudaFree(out);
    return (e == cudaSuccess && cudaGetLastError() == cudaSuccess) ? 0 : -3;
}

}  // extern "C"
