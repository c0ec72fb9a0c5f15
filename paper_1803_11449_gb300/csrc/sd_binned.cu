// sd_binned.cu -- Algorithm 1 (Update DHLA) by binning: the bit-sets of a
// chunk of pairs are sorted by the DHLA slice they fall in, then each slice
// is updated in shared memory by one block.
//
// Why: a pair sets r bits per direction at unrelated places in a DHLA of
// tens of MiB.  Done in place, every bit-set is a random L2 operation and
// the update runs at the L2's random-operation rate (about 2e11/s on GB300),
// far below the HBM stream rate of the pairs.  Here the same bit-sets become
// two streaming passes over a scratch buffer plus shared-memory atomics:
//
//   k_bin    reads a tile of pairs, computes every bit-set (word w, bit b),
//            counts them per slice (slice = w >> slice_log2, a block's worth
//            of shared memory), sorts them by slice in shared memory and
//            appends each slice's run to that slice's bin in one coalesced
//            write.  Entries are (w mod 2^slice_log2) << 5 | b.
//   k_apply  one block per slice (taken from a work counter): ORs the bin's
//            entries into a shared-memory copy of the slice, then ORs the
//            slice into the DHLA with plain loads and stores (no other block
//            touches that slice during the launch).
//
// A bin that is full falls back to a relaxed red.or on the DHLA word for the
// entries that do not fit: correct in either case, because every step only
// ORs bits in.  The result equals Algorithm 1's DHLA bit for bit.
#include "sd_common.cuh"

namespace sd {


// Constants of one direction, picked with selects rather than by indexing
// the kernel parameter with a run-time direction (that would copy the whole
// parameter block to local memory).
struct DirConst {
    uint32_t A0;
    uint64_t A1, B1;
    uint64_t base;  // first word of the direction
};

__device__ __forceinline__ DirConst dir_const(const Geometry &G, uint32_t d) {
    DirConst c;
    c.A0 = d ? G.h[1].A0 : G.h[0].A0;
    c.A1 = d ? G.h[1].A1 : G.h[0].A1;
    c.B1 = d ? G.h[1].B1 : G.h[0].B1;
    c.base = d ? G.dir_words : 0ull;
    return c;
}

__device__ __forceinline__ uint64_t bit_word(const Geometry &G, const DirConst &c, uint32_t i, uint32_t key,
                                             uint32_t c0, uint32_t b) {
    const uint32_t ci = (i == 0) ? c0 : dh_row(G, i, key, c0);
    return c.base + (uint64_t)i * G.row_words + (uint64_t)ci * G.wpc + (b >> 5);
}

// Shared memory of k_bin: tile pairs (2 words each), per-update (slice,
// rank), the slice-sorted entries, and per-slice histogram / offsets / bases.
__global__ void __launch_bounds__(512)
k_bin(const uint32_t *__restrict__ pairs, uint64_t n, uint32_t *__restrict__ grid, Geometry G, BinArgs B) {
    extern __shared__ uint32_t sm[];
    const uint32_t TP = B.tile_pairs;
    const uint32_t upd_per_pair = G.dirs * G.r;
    const uint32_t U = TP * upd_per_pair;  // bit-sets per tile
    uint32_t *spairs = sm;                 // [2*TP]
    uint32_t *meta = spairs + 2 * TP;      // [U]: slice << 20 | rank
    uint32_t *sorted = meta + U;           // [U]
    uint32_t *hist = sorted + U;           // [S]
    uint32_t *offs = hist + B.S;           // [S]
    uint32_t *base = offs + B.S;           // [S]
    __shared__ uint32_t warp_tot[32];

    for (uint32_t s = threadIdx.x; s < B.S; s += blockDim.x) hist[s] = 0;
    const uint64_t ntiles = (n + TP - 1) / TP;
    const uint32_t lane = threadIdx.x & 31u, wid = threadIdx.x >> 5, nwarps = blockDim.x >> 5;
    const uint32_t smask = (1u << B.slice_log2) - 1u;

    for (uint64_t t = blockIdx.x; t < ntiles; t += gridDim.x) {
        const uint64_t p0 = t * TP;
        const uint32_t np = (uint32_t)((n - p0) < TP ? (n - p0) : TP);
        __syncthreads();  // previous tile fully written out; hist is zero
        for (uint32_t q = threadIdx.x; q < 2 * np; q += blockDim.x) spairs[q] = ld_stream_u32(pairs + 2 * p0 + q);
        __syncthreads();
        // pass 1: slice of every bit-set and its rank inside the slice.
        // Update (d, i) of pair p is stored at meta[(d*r + i)*TP + p].
        for (uint32_t p = threadIdx.x; p < np; p += blockDim.x) {
            const uint32_t src = spairs[2 * p], dst = spairs[2 * p + 1];
            for (uint32_t d = 0; d < G.dirs; d++) {
                const DirConst c = dir_const(G, d);
                const uint32_t key = d ? dst : src, elem = d ? src : dst;
                const uint32_t b = (uint32_t)((c.A1 * (uint64_t)elem + c.B1) >> (64u - G.lg));
                const uint32_t c0 = dh0(c.A0, G.k, key);
                for (uint32_t i = 0; i < G.r; i++) {
                    const uint32_t s = (uint32_t)(bit_word(G, c, i, key, c0, b) >> B.slice_log2);
                    meta[(d * G.r + i) * TP + p] = (s << 20) | atomicAdd(&hist[s], 1u);
                }
            }
        }
        __syncthreads();
        // exclusive scan of hist into offs; reserve each slice's run in its bin
        {
            const uint32_t per = (B.S + blockDim.x - 1) / blockDim.x;
            const uint32_t s0 = threadIdx.x * per, s1 = min(s0 + per, B.S);
            uint32_t cnt = 0;
            for (uint32_t s = s0; s < s1; s++) cnt += hist[s];
            uint32_t incl = cnt;
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const uint32_t v = __shfl_up_sync(0xFFFFFFFFu, incl, o);
                if ((int)lane >= o) incl += v;
            }
            if (lane == 31) warp_tot[wid] = incl;
            __syncthreads();
            if (wid == 0) {
                uint32_t x = lane < nwarps ? warp_tot[lane] : 0;
#pragma unroll
                for (int o = 1; o < 32; o <<= 1) {
                    const uint32_t v = __shfl_up_sync(0xFFFFFFFFu, x, o);
                    if ((int)lane >= o) x += v;
                }
                if (lane < nwarps) warp_tot[lane] = x;
            }
            __syncthreads();
            uint32_t run = incl - cnt + (wid ? warp_tot[wid - 1] : 0);
            for (uint32_t s = s0; s < s1; s++) {
                offs[s] = run;
                run += hist[s];
                base[s] = hist[s] ? atomicAdd(&B.count[s], hist[s]) : 0u;
            }
        }
        __syncthreads();
        // pass 2: place every entry at its slice's offset + rank
        for (uint32_t p = threadIdx.x; p < np; p += blockDim.x) {
            const uint32_t src = spairs[2 * p], dst = spairs[2 * p + 1];
            for (uint32_t d = 0; d < G.dirs; d++) {
                const DirConst c = dir_const(G, d);
                const uint32_t key = d ? dst : src, elem = d ? src : dst;
                const uint32_t b = (uint32_t)((c.A1 * (uint64_t)elem + c.B1) >> (64u - G.lg));
                const uint32_t c0 = dh0(c.A0, G.k, key);
                for (uint32_t i = 0; i < G.r; i++) {
                    const uint64_t w = bit_word(G, c, i, key, c0, b);
                    const uint32_t m = meta[(d * G.r + i) * TP + p];
                    sorted[offs[m >> 20] + (m & 0xFFFFFu)] = (((uint32_t)w & smask) << 5) | (b & 31u);
                }
            }
        }
        __syncthreads();
        // write-out: one warp per slice run, coalesced; overflow -> red.or
        for (uint32_t s = wid; s < B.S; s += nwarps) {
            const uint32_t len = hist[s];
            if (!len) continue;
            const uint32_t o = offs[s], bs = base[s];
            for (uint32_t k = lane; k < len; k += 32) {
                const uint32_t e = sorted[o + k];
                if (bs + k < B.cap) {
                    B.bins[(uint64_t)s * B.cap + bs + k] = e;
                } else {
                    const uint64_t w = ((uint64_t)s << B.slice_log2) | (e >> 5);
                    red_or(grid + w, 1u << (e & 31u));
                }
            }
            __syncwarp();
            if (lane == 0) hist[s] = 0;
        }
    }
}

__global__ void __launch_bounds__(1024)
k_apply(uint32_t *__restrict__ grid, BinArgs B) {
    extern __shared__ uint32_t slice[];
    __shared__ uint32_t s_cur;
    const uint32_t SW = 1u << B.slice_log2;
    for (;;) {
        __syncthreads();
        if (threadIdx.x == 0) s_cur = atomicAdd(B.work, 1u);
        __syncthreads();
        const uint32_t s = s_cur;
        if (s >= B.S) break;
        uint4 *s4 = reinterpret_cast<uint4 *>(slice);
        for (uint32_t i = threadIdx.x; i < SW / 4; i += blockDim.x) s4[i] = make_uint4(0, 0, 0, 0);
        __syncthreads();
        const uint32_t cnt = min(B.count[s], B.cap);
        const uint32_t *bin = B.bins + (uint64_t)s * B.cap;
        // entries: 16-byte loads where aligned (cap is a multiple of 4)
        for (uint32_t q = threadIdx.x; q < cnt / 4; q += blockDim.x) {
            const uint4 e = ld_stream_v4(reinterpret_cast<const uint4 *>(bin) + q);
            atomicOr(&slice[e.x >> 5], 1u << (e.x & 31u));
            atomicOr(&slice[e.y >> 5], 1u << (e.y & 31u));
            atomicOr(&slice[e.z >> 5], 1u << (e.z & 31u));
            atomicOr(&slice[e.w >> 5], 1u << (e.w & 31u));
        }
        for (uint32_t q = (cnt & ~3u) + threadIdx.x; q < cnt; q += blockDim.x) {
            const uint32_t e = ld_stream_u32(bin + q);
            atomicOr(&slice[e >> 5], 1u << (e & 31u));
        }
        __syncthreads();
        // OR the slice into the DHLA (this block is the slice's only writer)
        const uint64_t w0 = (uint64_t)s << B.slice_log2;
        const uint64_t left = B.total_words - w0;
        const uint32_t words = left < (uint64_t)SW ? (uint32_t)left : SW;
        uint4 *g4 = reinterpret_cast<uint4 *>(grid + w0);
        for (uint32_t i = threadIdx.x; i < words / 4; i += blockDim.x) {
            const uint4 v = s4[i];
            if (v.x | v.y | v.z | v.w) {
                uint4 g = g4[i];
                g.x |= v.x; g.y |= v.y; g.z |= v.z; g.w |= v.w;
                g4[i] = g;
            }
        }
        if (threadIdx.x == 0) B.count[s] = 0;
    }
}

__global__ void k_zero_u32(uint32_t *p, uint32_t n) {
    for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) p[i] = 0;
}

size_t bin_smem_bytes(uint32_t tile_pairs, uint32_t upd_per_pair, uint32_t S) {
    return ((size_t)2 * tile_pairs + 2ull * tile_pairs * upd_per_pair + 3ull * S) * 4;
}

// One chunk: bin then apply.  `scratch` holds bins, counts and the work
// counter as laid out by the caller (see BinLayout in the API).
cudaError_t launch_binned_chunk(const uint32_t *pairs, uint64_t n, uint32_t *grid, const Geometry &G,
                                const BinArgs &B, int num_sms, cudaStream_t s) {
    const size_t smem_bin = bin_smem_bytes(B.tile_pairs, G.dirs * G.r, B.S);
    const size_t smem_apply = (size_t)4 << B.slice_log2;
    cudaError_t e = cudaFuncSetAttribute(k_bin, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem_bin);
    if (e != cudaSuccess) return e;
    e = cudaFuncSetAttribute(k_apply, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem_apply);
    if (e != cudaSuccess) return e;
    int per_sm = 0;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_bin, 512, smem_bin);
    if (e != cudaSuccess) return e;
    const uint64_t tiles = (n + B.tile_pairs - 1) / B.tile_pairs;
    uint64_t blocks = (uint64_t)num_sms * (per_sm > 0 ? per_sm : 1);
    if (tiles < blocks) blocks = tiles ? tiles : 1;
    k_bin<<<(unsigned)blocks, 512, smem_bin, s>>>(pairs, n, grid, G, B);
    e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    k_zero_u32<<<1, 32, 0, s>>>(B.work, 1);
    int per_sm_a = 0;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm_a, k_apply, 1024, smem_apply);
    if (e != cudaSuccess) return e;
    uint64_t ablocks = (uint64_t)num_sms * (per_sm_a > 0 ? per_sm_a : 1);
    if (B.S < ablocks) ablocks = B.S;
    k_apply<<<(unsigned)ablocks, 1024, smem_apply, s>>>(grid, B);
    return cudaGetLastError();
}

}  // namespace sd
