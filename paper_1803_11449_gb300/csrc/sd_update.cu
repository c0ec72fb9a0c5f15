// sd_update.cu -- Algorithm 1 (Update DHLA) over a stream of (src, dst)
// pairs, one launch per sd_update call.
//
// Design (GB300): the pair stream is read once from HBM with 16-byte
// streaming loads (two pairs per load, `unroll` loads in flight per thread);
// both hashes are computed in registers; the r bit-sets per direction go to
// the L2-resident DHLA as relaxed `red.or` reductions.  Mode 1 adds
// Algorithm 1's own test ("if the bit is 1, continue") as a weak cached load
// so set bits cost a load instead of an atomic; mode 2 additionally merges
// bit-sets that hit the same word inside a warp (__match_any_sync).  Modes 3
// and 4 put a shared-memory filter of words known to be set in front of the
// test (3) or of the plain reduction (4): with Zipf-distributed hosts most
// bit-sets repeat bits that heavy hosts set long ago, and those never leave
// the SM.  The grid is persistent: a multiple of the SM count, grid-stride
// over the pairs with a trip count that is uniform across each warp (mode 2
// needs converged warps).
#include "sd_common.cuh"

namespace sd {

// Per-block filter of DHLA words with bits known to be set: a direct-mapped
// table in shared memory of 64-bit entries (word index << 32 | known mask).
// An entry is written with one 64-bit store, so a reader always sees a tag
// and a mask that belong together; every bit in a stored mask is either
// already 1 in the DHLA or covered by a reduction this block has issued, and
// those complete before the kernel ends.  So a filter hit may skip the
// bit-set; a lost or overwritten entry only costs a redundant operation.
struct Filter {
    unsigned long long *tab;
    uint32_t shift;  // 32 - log2(entries)
};

__device__ __forceinline__ uint32_t filter_slot(const Filter &f, uint32_t word) {
    return (word * 0x9E3779B1u) >> f.shift;
}

// Set bit H1(elem) of the estimators DH_i(key), i < R, of one direction.
// `word0` is the index of the direction's first DHLA word (filter tags).
template <int R, int MODE>
__device__ __forceinline__ void set_bits(uint32_t *__restrict__ dgrid, const Geometry &G,
                                         const HashDir &h, uint32_t key, uint32_t elem,
                                         bool valid, const Filter &f, uint32_t word0) {
    const uint32_t bit = h1(h, G.lg, elem);
    const uint32_t c0 = dh0(h.A0, G.k, key);
    const uint32_t mask = 1u << (bit & 31u);
    uint32_t *const base = dgrid + (bit >> 5);
    uint32_t *addr[R];
    uint32_t widx[R];
#pragma unroll
    for (int i = 0; i < R; i++) {
        const uint32_t ci = (i == 0) ? c0 : dh_row(G, i, key, c0);
        const uint64_t off = (uint64_t)i * G.row_words + (uint64_t)ci * G.wpc;
        addr[i] = base + off;
        widx[i] = word0 + (uint32_t)off + (bit >> 5);
    }
    if (MODE >= 3) {
        // filter first; then test (mode 3) or reduce directly (mode 4)
        unsigned long long e[R];
#pragma unroll
        for (int i = 0; i < R; i++) e[i] = valid ? f.tab[filter_slot(f, widx[i])] : 0ull;
        bool need[R];
#pragma unroll
        for (int i = 0; i < R; i++) {
            const bool tag_ok = (uint32_t)(e[i] >> 32) == widx[i];
            need[i] = valid && !(tag_ok && ((uint32_t)e[i] & mask));
        }
        uint32_t cur[R];
#pragma unroll
        for (int i = 0; i < R; i++) cur[i] = (MODE == 3 && need[i]) ? ld_weak(addr[i]) : 0u;
#pragma unroll
        for (int i = 0; i < R; i++) {
            if (!need[i]) continue;
            if (!(cur[i] & mask)) red_or(addr[i], mask);
            const bool tag_ok = (uint32_t)(e[i] >> 32) == widx[i];
            const uint32_t known = (tag_ok ? (uint32_t)e[i] : 0u) | cur[i] | mask;
            f.tab[filter_slot(f, widx[i])] = ((unsigned long long)widx[i] << 32) | known;
        }
        return;
    }
    if (MODE == 0) {
        if (valid) {
#pragma unroll
            for (int i = 0; i < R; i++) red_or(addr[i], mask);
        }
    } else if (MODE == 1) {
        uint32_t cur[R];
#pragma unroll
        for (int i = 0; i < R; i++) cur[i] = valid ? ld_weak(addr[i]) : mask;
#pragma unroll
        for (int i = 0; i < R; i++)
            if (!(cur[i] & mask)) red_or(addr[i], mask);
    } else {
        const uint32_t lane = threadIdx.x & 31u;
        uint32_t cur[R];
#pragma unroll
        for (int i = 0; i < R; i++) cur[i] = valid ? ld_weak(addr[i]) : mask;
#pragma unroll
        for (int i = 0; i < R; i++) {
            const bool need = !(cur[i] & mask);
            // lanes that need the same word form one group; the lowest lane
            // ORs the group's masks and issues a single reduction
            const unsigned peers =
                __match_any_sync(0xFFFFFFFFu, need ? (unsigned long long)(uintptr_t)addr[i] : 0ull);
            if (need) {
                uint32_t m = 0;
                unsigned rest = peers;
                while (rest) {
                    const int src = __ffs(rest) - 1;
                    rest &= rest - 1u;
                    m |= __shfl_sync(peers, mask, src);
                }
                if ((int)lane == __ffs(peers) - 1) red_or(addr[i], m);
            }
        }
    }
}

template <int R, int MODE>
__device__ __forceinline__ void apply_pair(uint32_t *__restrict__ grid, const Geometry &G,
                                           uint32_t src, uint32_t dst, bool valid, const Filter &f) {
    set_bits<R, MODE>(grid, G, G.h[0], src, dst, valid, f, 0u);
    if (G.dirs > 1)
        set_bits<R, MODE>(grid + G.dir_words, G, G.h[1], dst, src, valid, f, (uint32_t)G.dir_words);
}

// pairs: 8-byte aligned (the launcher guarantees it).  The first pair is
// handled alone when needed to reach 16-byte alignment, then 2 pairs per
// 16-byte load, then a last odd pair.
template <int R, int MODE, int UNROLL>
__global__ void __launch_bounds__(1024)
k_update(const uint32_t *__restrict__ pairs, uint64_t n, uint32_t *__restrict__ grid, Geometry G,
         uint32_t filter_log2) {
    extern __shared__ unsigned long long filter_tab[];
    Filter f{filter_tab, 32u - filter_log2};
    if (MODE >= 3) {
        // empty entries carry the tag 0xFFFFFFFF, never a word index (the
        // launcher only enables the filter when the DHLA has fewer words)
        for (uint32_t i = threadIdx.x; i < (1u << filter_log2); i += blockDim.x)
            filter_tab[i] = 0xFFFFFFFF00000000ull;
        __syncthreads();
    }
    const uint64_t tid = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
    const uint64_t head = (((uintptr_t)pairs & 15u) != 0 && n > 0) ? 1 : 0;
    const uint4 *body = reinterpret_cast<const uint4 *>(pairs + 2 * head);
    const uint64_t nv = (n - head) / 2;
    const uint64_t tail = head + 2 * nv;  // index of a last odd pair, if tail < n

    // head and tail pairs: processed by the first warp of block 0, converged
    if (blockIdx.x == 0 && threadIdx.x < 32) {
        const bool h_ok = (threadIdx.x == 0) && head;
        const bool t_ok = (threadIdx.x == 1) && (tail < n);
        const uint64_t at = h_ok ? 0 : (t_ok ? tail : 0);
        uint32_t s = 0, d = 0;
        if (h_ok || t_ok) {
            s = pairs[2 * at];
            d = pairs[2 * at + 1];
        }
        apply_pair<R, MODE>(grid, G, s, d, h_ok || t_ok, f);
    }

    const uint64_t step = stride * UNROLL;
    const uint64_t iters = (nv + step - 1) / step;  // identical for every thread
    for (uint64_t it = 0; it < iters; it++) {
        uint4 q[UNROLL];
        bool ok[UNROLL];
#pragma unroll
        for (int u = 0; u < UNROLL; u++) {
            const uint64_t v = it * step + (uint64_t)u * stride + tid;
            ok[u] = v < nv;
            q[u] = ok[u] ? ld_stream_v4(body + v) : make_uint4(0, 0, 0, 0);
        }
#pragma unroll
        for (int u = 0; u < UNROLL; u++) {
            apply_pair<R, MODE>(grid, G, q[u].x, q[u].y, ok[u], f);
            apply_pair<R, MODE>(grid, G, q[u].z, q[u].w, ok[u], f);
        }
    }
}

// Pairs that are only 4-byte aligned (an odd word offset): one pair per
// thread with 32-bit loads.  Correct for any alignment; not tuned.
template <int R>
__global__ void __launch_bounds__(256)
k_update_unaligned(const uint32_t *__restrict__ pairs, uint64_t n, uint32_t *__restrict__ grid,
                   Geometry G) {
    const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
    const Filter f{nullptr, 0};
    for (uint64_t t = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; t < n; t += stride)
        apply_pair<R, 0>(grid, G, ld_stream_u32(pairs + 2 * t), ld_stream_u32(pairs + 2 * t + 1), true, f);
}

template <int R, int MODE, int UNROLL>
static cudaError_t launch3(const uint32_t *pairs, uint64_t n, uint32_t *grid, const Geometry &G,
                           const Tuning &T, int num_sms, cudaStream_t s) {
    auto kern = k_update<R, MODE, UNROLL>;
    const uint32_t flog = MODE >= 3 ? T.filter_log2 : 0u;
    const size_t smem = MODE >= 3 ? ((size_t)8 << flog) : 0;
    int per_sm = 0;
    cudaError_t e = prepare_launch(reinterpret_cast<const void *>(kern), (int)T.block_threads, smem, &per_sm);
    if (e != cudaSuccess) return e;
    if (per_sm < 1) per_sm = 1;
    const int want = T.blocks_per_sm ? (int)T.blocks_per_sm : per_sm;
    const int bps = want < per_sm ? want : per_sm;
    // never more blocks than needed to give every thread one 16-byte load
    const uint64_t loads = n / 2 + 1;
    uint64_t blocks = (uint64_t)num_sms * bps;
    const uint64_t need = (loads + T.block_threads - 1) / T.block_threads;
    if (need < blocks) blocks = need > 0 ? need : 1;
    kern<<<(unsigned)blocks, T.block_threads, smem, s>>>(pairs, n, grid, G, flog);
    return cudaGetLastError();
}

template <int R, int MODE>
static cudaError_t launch2(const uint32_t *pairs, uint64_t n, uint32_t *grid, const Geometry &G,
                           const Tuning &T, int num_sms, cudaStream_t s) {
    switch (T.unroll) {
        case 1: return launch3<R, MODE, 1>(pairs, n, grid, G, T, num_sms, s);
        case 4: return launch3<R, MODE, 4>(pairs, n, grid, G, T, num_sms, s);
        default: return launch3<R, MODE, 2>(pairs, n, grid, G, T, num_sms, s);
    }
}

template <int R>
static cudaError_t launch1(const uint32_t *pairs, uint64_t n, uint32_t *grid, const Geometry &G,
                           const Tuning &T, int num_sms, cudaStream_t s) {
    if (((uintptr_t)pairs & 7u) != 0) {
        const uint64_t blocks64 = (n + 255) / 256;
        const unsigned blocks = (unsigned)(blocks64 < (uint64_t)num_sms * 8 ? (blocks64 ? blocks64 : 1)
                                                                           : (uint64_t)num_sms * 8);
        k_update_unaligned<R><<<blocks, 256, 0, s>>>(pairs, n, grid, G);
        return cudaGetLastError();
    }
    uint32_t mode = T.mode;
    // the filter tags words with 32-bit indices; 0xFFFFFFFF marks empty slots
    if (mode >= 3 && (uint64_t)G.dirs * G.dir_words >= 0xFFFFFFFFull) mode = 1;
    switch (mode) {
        case 1: return launch2<R, 1>(pairs, n, grid, G, T, num_sms, s);
        case 2: return launch2<R, 2>(pairs, n, grid, G, T, num_sms, s);
        case 3: return launch2<R, 3>(pairs, n, grid, G, T, num_sms, s);
        case 4: return launch2<R, 4>(pairs, n, grid, G, T, num_sms, s);
        default: return launch2<R, 0>(pairs, n, grid, G, T, num_sms, s);
    }
}

cudaError_t launch_update(const uint32_t *pairs, uint64_t n, uint32_t *grid, const Geometry &G,
                          const Tuning &T, int num_sms, cudaStream_t s) {
    if (n == 0) return cudaSuccess;
    switch (G.r) {
        case 3: return launch1<3>(pairs, n, grid, G, T, num_sms, s);
        case 4: return launch1<4>(pairs, n, grid, G, T, num_sms, s);
        case 5: return launch1<5>(pairs, n, grid, G, T, num_sms, s);
        case 6: return launch1<6>(pairs, n, grid, G, T, num_sms, s);
        case 7: return launch1<7>(pairs, n, grid, G, T, num_sms, s);
        case 8: return launch1<8>(pairs, n, grid, G, T, num_sms, s);
        default: return cudaErrorInvalidValue;
    }
}

}  // namespace sd
