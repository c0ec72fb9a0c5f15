// sd_close.cu -- the window-close path (Algorithm 2 and the estimation step
// of §4.2) on the GPU.
//
//   k_row_stats   z_0 = g - popcount for every estimator, ZR(i) per row, the
//                 hot bitmap of each row (z_0 <= zhot, i.e. z_0 < Zmin) and
//                 |HE(i)|.
//   k_compact     sorted lists HE(0) and HE(1) (all HE(i) for the staged
//                 join of sd_join.cu) from their bitmaps.
//   k_restore     the candidate set K = {a : DH_i(a) in HE(i) for all i}.
//   k_estimate    SZ(a) from ULE(a) = AND of a's r estimators (16-byte
//                 chunks, several candidates per warp), keeping (a, SZ) when
//                 SZ <= szmax.
//   k_sort_small  orders each direction's hits by address (bitonic, smem).
//   k_ss_*        the same for up to 2^19 hits: a sample sort (splitters
//                 from a sorted sample, keys scattered to buckets, each
//                 bucket sorted by one block).
//   k_sort_segments + k_merge_rank  longer lists, or a sample sort that fell
//                 short: sorted 2048-key segments, then pairwise merges.
//   k_reset       clears the DHLA and the per-window counters.
//   k_merge_or    dst |= src over whole DHLAs (multi-monitor merge).
//   k_*_many      the same kernels over an array of windows of one shape
//                 (sd_close_many): one launch per phase for all of them.
//
// Restore.  The paper's GPU restore (Algorithms 3 and 4) joins HE(0) x HE(1)
// x HE(2) and extends the surviving partial addresses row by row.  Here the
// join stops after HE(0) x HE(1): with c0 = DH_0(a) and c1 = DH_1(a),
// L = c0 xor c1 is the low k bits of a (Eq. 3 for i = 1), and because
// DH_0(a) = (A0 a mod 2^32) >> (32-k) with A0 odd, the remaining 32-k high
// bits H of a follow from c0 by one multiplication with A0^-1:
//   write A0*L mod 2^32 = Qh*2^k + Ql; then A0*a mod 2^32 = u*2^k + Ql with
//   u = (A0*H + Qh) mod 2^(32-k), and DH_0(a) = c0 fixes u:
//     k >= 16: u = c0 >> (2k-32), provided (Ql >> (32-k)) equals the low
//              2k-32 bits of c0 (otherwise no a exists);
//     k <  16: u = (c0 << (32-2k)) | t for each t < 2^(32-2k).
//   H = A0^-1 (u - Qh) mod 2^(32-k),  a = H*2^k + L.
// Each a found this way has DH_0(a) = c0 and DH_1(a) = c1 by construction and
// is kept when DH_i(a) is hot for i = 2..r-1: exactly K.  The work is
// |HE(0)|*|HE(1)|*2^max(0,32-2k) cheap integer tests instead of a join whose
// intermediate lists grow with |HE|^3.
#include <algorithm>

#include "sd_common.cuh"

namespace sd {

__device__ __forceinline__ uint32_t warp_sum(uint32_t v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xFFFFFFFFu, v, o);
    return v;
}

// ------------------------------------------------------------- row stats
// One thread per estimator; a warp covers 32 consecutive estimators of one
// row (2^k >= 32 because (r-1)k >= (r-2)alpha + k >= 32 with r <= 8).
__device__ __forceinline__ void row_stats_body(const uint32_t *__restrict__ grid, const Geometry &G, int zhot,
                                               uint32_t *__restrict__ hotmap, StatBlock *__restrict__ st,
                                               uint32_t bx, uint32_t nbx) {
    __shared__ unsigned long long s_zr[2 * kMaxRows];
    __shared__ unsigned s_nhot[2 * kMaxRows];
    if (threadIdx.x < 2 * kMaxRows) {
        s_zr[threadIdx.x] = 0;
        s_nhot[threadIdx.x] = 0;
    }
    __syncthreads();
    const uint64_t ncell = (uint64_t)G.dirs * G.r << G.k;
    const uint64_t stride = (uint64_t)nbx * blockDim.x;
    const uint32_t lane = threadIdx.x & 31u;
    for (uint64_t q = (uint64_t)bx * blockDim.x + threadIdx.x; q < ncell; q += stride) {
        const uint32_t *cell = grid + q * G.wpc;
        uint32_t pop = 0;
        if ((G.wpc & 3u) == 0) {
            const uint4 *c4 = reinterpret_cast<const uint4 *>(cell);
            for (uint32_t w = 0; w < G.wpc / 4; w++) {
                const uint4 v = __ldg(c4 + w);
                pop += __popc(v.x) + __popc(v.y) + __popc(v.z) + __popc(v.w);
            }
        } else {
            for (uint32_t w = 0; w < G.wpc; w++) pop += __popc(__ldg(cell + w));
        }
        const uint32_t z0 = G.g - pop;
        const unsigned hot = __ballot_sync(0xFFFFFFFFu, (int)z0 <= zhot);
        const uint32_t zsum = warp_sum(z0);
        if (lane == 0) {
            const uint32_t row = (uint32_t)(q >> G.k);  // dir * r + i
            hotmap[q >> 5] = hot;
            atomicAdd(&s_zr[row], (unsigned long long)zsum);
            atomicAdd(&s_nhot[row], (unsigned)__popc(hot));
        }
    }
    __syncthreads();
    // one global atomic per block and row
    for (uint32_t row = threadIdx.x; row < G.dirs * G.r; row += blockDim.x) {
        const uint32_t d = row / G.r, i = row % G.r;
        if (s_zr[row]) atomicAdd(&st->zr[d][i], s_zr[row]);
        if (s_nhot[row]) atomicAdd(&st->nhot[d][i], s_nhot[row]);
    }
}

__global__ void __launch_bounds__(256)
k_row_stats(const uint32_t *__restrict__ grid, Geometry G, int zhot, uint32_t *__restrict__ hotmap,
            StatBlock *__restrict__ st) {
    row_stats_body(grid, G, zhot, hotmap, st, blockIdx.x, gridDim.x);
}

// ---------------------------------------------------------------- compact
// One block per (dir, row in {0, 1}): HE(row) in ascending order.
__device__ __forceinline__ void compact_body(const uint32_t *__restrict__ hotmap, const Geometry &G,
                                             uint32_t *__restrict__ he, uint32_t rows, uint32_t bx) {
    const uint32_t dir = bx / rows, row = bx % rows;
    const uint32_t nw = (1u << G.k) >> 5;
    const uint32_t *bm = hotmap + ((uint64_t)dir * G.r + row) * nw;
    uint32_t *out = he + ((uint64_t)dir * rows + row) * (1ull << G.k);
    const uint32_t per = (nw + blockDim.x - 1) / blockDim.x;
    const uint32_t w0 = threadIdx.x * per;
    const uint32_t w1 = min(w0 + per, nw);
    uint32_t cnt = 0;
    for (uint32_t w = w0; w < w1; w++) cnt += __popc(bm[w]);
    // block exclusive scan of cnt
    __shared__ uint32_t warp_tot[32];
    const uint32_t lane = threadIdx.x & 31u, wid = threadIdx.x >> 5;
    uint32_t incl = cnt;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const uint32_t v = __shfl_up_sync(0xFFFFFFFFu, incl, o);
        if ((int)lane >= o) incl += v;
    }
    if (lane == 31) warp_tot[wid] = incl;
    __syncthreads();
    if (wid == 0) {
        const uint32_t nwarps = blockDim.x >> 5;
        uint32_t t = lane < nwarps ? warp_tot[lane] : 0;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const uint32_t v = __shfl_up_sync(0xFFFFFFFFu, t, o);
            if ((int)lane >= o) t += v;
        }
        if (lane < nwarps) warp_tot[lane] = t;  // inclusive over warps
    }
    __syncthreads();
    uint32_t pos = incl - cnt + (wid ? warp_tot[wid - 1] : 0);
    for (uint32_t w = w0; w < w1; w++) {
        uint32_t b = bm[w];
        while (b) {
            const uint32_t bit = __ffs(b) - 1;
            b &= b - 1u;
            out[pos++] = (w << 5) | bit;
        }
    }
}

__global__ void __launch_bounds__(1024)
k_compact(const uint32_t *__restrict__ hotmap, Geometry G, uint32_t *__restrict__ he, uint32_t rows) {
    compact_body(hotmap, G, he, rows, blockIdx.x);
}

// ---------------------------------------------------------------- restore
__device__ __forceinline__ bool hot_at(const uint32_t *bm_row, uint32_t c) {
    return (bm_row[c >> 5] >> (c & 31u)) & 1u;
}

constexpr uint32_t kRestoreTileMax = 256;  // c0 values per k_restore tile

// Per-warp output buffers of k_restore: candidates and hits are reserved in
// the global lists 32 at a time (one atomic per flush instead of one per
// finding warp, which serialised on the two counters).
constexpr int kWarpBuf = 64;

__device__ __forceinline__ void flush_cands(const RestoreArgs &A, uint32_t dir, uint32_t *cbuf, uint32_t &ccount,
                                            uint32_t lane) {
    if (ccount == 0) return;
    unsigned long long base = 0;
    if (lane == 0) base = atomicAdd(&A.stats->ncand[dir], (unsigned long long)ccount);
    base = __shfl_sync(0xFFFFFFFFu, base, 0);
    for (uint32_t q = lane; q < ccount; q += 32)
        if (base + q < A.cand_cap) A.cand[(uint64_t)dir * A.cand_cap + base + q] = cbuf[q];
    ccount = 0;
    __syncwarp();
}

__device__ __forceinline__ void flush_hits(const RestoreArgs &A, uint32_t dir, unsigned long long *hbuf,
                                           uint32_t &hcount, uint32_t lane) {
    if (hcount == 0) return;
    unsigned long long base = 0;
    if (lane == 0) base = atomicAdd(&A.stats->nhits[dir], (unsigned long long)hcount);
    base = __shfl_sync(0xFFFFFFFFu, base, 0);
    for (uint32_t q = lane; q < hcount; q += 32)
        if (base + q < A.hits_cap) A.hits[(uint64_t)dir * A.hits_cap + base + q] = hbuf[q];
    hcount = 0;
    __syncwarp();
}

// 32-bit load from shared memory at byte address `addr`.
__device__ __forceinline__ uint32_t lds_u32(uint32_t addr) {
    uint32_t v;
    asm volatile("ld.shared.u32 %0, [%1];" : "=r"(v) : "r"(addr));
    return v;
}

// One (c0, c1) test for k >= 16 and R rows, the hot bitmap rows 2..R-1 in
// shared memory at byte address hot2s (row i - 2 at + (i - 2) nw 4): a's low
// k bits are L = c0 ^ c1; its high 32 - k bits are A0^-1 (c0 >> (2k - 32) -
// (A0 L >> k)) mod 2^(32-k), computed as one multiply by A0^-1 2^k; unless
// k = 16, the low 2k - 32 bits of c0 must also match the top bits of A0 L
// mod 2^k.  Returns whether a is in K; a is set.
template <int R, bool K16, int ALPHA>
__device__ __forceinline__ bool restore_test(uint32_t c0, uint32_t c1, uint32_t k, uint32_t kmask, uint32_t lowbits,
                                             uint32_t lowmask, uint32_t A0, uint32_t A0inv_k, uint32_t hot2s,
                                             uint32_t nw4, const uint32_t (&sh)[R > 2 ? R - 2 : 1], uint32_t &a) {
    const uint32_t L = c0 ^ c1;
    const uint32_t Q = A0 * L;
    uint32_t found = 1u;
    if (K16) {
        a = A0inv_k * (c0 - (Q >> 16)) + L;
    } else {
        a = A0inv_k * ((c0 >> lowbits) - (Q >> k)) + L;
        found = ((Q & kmask) >> (32u - k)) == (c0 & lowmask);
    }
#pragma unroll
    for (int i = 2; i < R; i++) {
        // with k = 16 and a compile-time alpha the shifts and masks are constants
        const uint32_t s = ALPHA ? (uint32_t)((i - 1) * ALPHA) : sh[i - 2];
        const uint32_t m = K16 ? 0xFFFFu : kmask;
        const uint32_t ci = (ALPHA && s >= 32u ? 0u : (ALPHA ? (a >> (s & 31u)) : shr_clamp(a, s))) & m ^ c0;
        const uint32_t word = lds_u32(hot2s + (uint32_t)(i - 2) * nw4 + ((ci >> 3) & ~3u));
        found &= word >> (ci & 31u);
    }
    return found & 1u;
}

// The tests of two c1 values per thread against the tile's c0 values, for
// k >= 16 with the hot bitmap in shared memory; candidates go to the warp's
// buffer.
template <int R, bool K16, int ALPHA>
__device__ __forceinline__ void restore_c1x2(const Geometry &G, const RestoreArgs &A, uint32_t dir,
                                             const uint32_t *s_c0, uint32_t nc0, uint32_t hot2s, uint32_t nw,
                                             uint32_t c1a, bool va, uint32_t c1b, bool vb, uint32_t A0,
                                             uint32_t A0inv, uint32_t *cbuf, uint32_t &ccount, uint32_t lane) {
    const uint32_t k = G.k, kmask = (1u << k) - 1u;
    const uint32_t lowbits = 2u * k - 32u, lowmask = (1u << lowbits) - 1u;
    const uint32_t A0inv_k = A0inv << k, nw4 = nw * 4u;
    uint32_t sh[R > 2 ? R - 2 : 1];
#pragma unroll
    for (int i = 2; i < R; i++) sh[i - 2] = (uint32_t)(i - 1) * G.alpha;
    const unsigned below = (1u << lane) - 1u;
    for (uint32_t q = 0; q < nc0; q++) {
        const uint32_t c0 = s_c0[q];  // same for the whole block
        uint32_t aa, ab;
        const bool fa = va && restore_test<R, K16, ALPHA>(c0, c1a, k, kmask, lowbits, lowmask, A0, A0inv_k, hot2s, nw4,
                                                           sh, aa);
        const bool fb = vb && restore_test<R, K16, ALPHA>(c0, c1b, k, kmask, lowbits, lowmask, A0, A0inv_k, hot2s, nw4,
                                                           sh, ab);
        const unsigned ba = __ballot_sync(0xFFFFFFFFu, fa), bb = __ballot_sync(0xFFFFFFFFu, fb);
        if (!(ba | bb)) continue;
        if (fa) cbuf[ccount + __popc(ba & below)] = aa;
        ccount += __popc(ba);
        if (fb) cbuf[ccount + __popc(bb & below)] = ab;
        ccount += __popc(bb);
        __syncwarp();
        if (ccount >= 32) flush_cands(A, dir, cbuf, ccount, lane);
    }
}

// Tiles t_begin, t_begin + t_step, ... below t_end of direction `dir`.
__device__ __forceinline__ void restore_body(const Geometry &G, const RestoreArgs &A, uint32_t dir, uint64_t t_begin,
                                             uint64_t t_end, uint64_t t_step) {
    extern __shared__ uint32_t smem[];
    __shared__ uint32_t s_cbuf[8][kWarpBuf];
    __shared__ uint32_t s_c0[kRestoreTileMax];
    __shared__ bool s_stop;
    __syncthreads();  // shared memory may still be in use by a previous call
    // per-direction scalars picked with selects: indexing the parameter
    // arrays with a run-time index would copy them to local memory
    if (!(dir ? A.run[1] : A.run[0])) return;
    const uint32_t n0 = dir ? A.n0[1] : A.n0[0];
    const uint32_t n1 = dir ? A.n1[1] : A.n1[0];
    if (n0 == 0 || n1 == 0) return;
    const uint32_t k = G.k, kmask = (1u << k) - 1u;
    const uint32_t hmask = (k >= 32u) ? 0u : ((1u << (32u - k)) - 1u);  // 32-k high bits
    const uint32_t nw = (1u << k) >> 5;
    const uint32_t A0 = dir ? G.h[1].A0 : G.h[0].A0;
    const uint32_t A0inv = dir ? G.h[1].A0inv : G.h[0].A0inv;
    const uint32_t *he0 = A.he + (uint64_t)dir * 2 * (1ull << k);
    const uint32_t *he1 = he0 + (1ull << k);
    const uint32_t *bm_dir = A.hotmap + (uint64_t)dir * G.r * nw;  // row i at bm_dir + i*nw
    const uint64_t J = (uint64_t)n1 << A.ulog;
    const uint32_t ntile0 = (n0 + A.tile0 - 1) / A.tile0;
    const uint64_t nchunk = (J + A.jchunk - 1) / A.jchunk;
    const uint64_t ntiles = (uint64_t)ntile0 * nchunk;
    const uint64_t t_stop = t_end < ntiles ? t_end : ntiles;
    if (t_begin >= t_stop) return;  // no tile of this direction for the block

    // rows 2..r-1 of the hot bitmap; row i is at hot2 + (i-2)*nw
    const uint32_t *hot2 = bm_dir + 2 * nw;
    if (A.smem_hot) {
        uint32_t *sb = smem;
        const uint32_t words = (G.r - 2) * nw;
        for (uint32_t w = threadIdx.x; w < words; w += blockDim.x) sb[w] = hot2[w];
        hot2 = sb;
        __syncthreads();
    }

    const uint32_t lane = threadIdx.x & 31u;
    uint32_t *cbuf = s_cbuf[threadIdx.x >> 5];
    uint32_t ccount = 0;  // warp-uniform
    const uint32_t lowbits = (k >= 16u) ? (2u * k - 32u) : 0u;
    const uint32_t lowmask = (1u << lowbits) - 1u;
    const uint32_t iters = A.jchunk / blockDim.x;  // jchunk is a multiple of blockDim
    // the specialised loop: k >= 16 (no enumeration of t), the hot bitmap in
    // shared memory, at most 8 rows, an even number of c1 steps
    const bool fast = k >= 16u && A.smem_hot && G.r <= 8u && (iters & 1u) == 0;
    const uint32_t hot2s = (uint32_t)__cvta_generic_to_shared(smem);

    for (uint64_t t = t_begin; t < t_stop; t += t_step) {
        const uint32_t t0 = (uint32_t)(t / nchunk);
        const uint64_t jc = t % nchunk;
        const uint32_t c0_base = t0 * A.tile0;
        const uint32_t nc0 = min(A.tile0, n0 - c0_base);
        __syncthreads();
        // once K has passed its capacity the direction reports nothing but
        // the overload, so the rest of its enumeration is skipped (one read
        // of the shared counter per tile, the same decision for the block)
        if (threadIdx.x == 0)
            s_stop = *reinterpret_cast<volatile unsigned long long *>(&A.stats->ncand[dir]) > A.cand_cap;
        for (uint32_t q = threadIdx.x; q < nc0; q += blockDim.x) s_c0[q] = he0[c0_base + q];
        __syncthreads();
        if (s_stop) break;
        if (fast) {
            // two c1 values per thread and step (iters is even: jchunk = 2 blockDim)
            for (uint32_t m = 0; m < iters; m += 2) {
                const uint64_t ja = jc * A.jchunk + (uint64_t)m * blockDim.x + threadIdx.x;
                const uint64_t jb = ja + blockDim.x;
                const bool va = ja < J, vb = jb < J;
                const uint32_t c1a = va ? he1[(uint32_t)ja] : 0u, c1b = vb ? he1[(uint32_t)jb] : 0u;
                if (G.r == 4u && k == 16u && G.alpha == 8u) {  // the core-link sketch
                    restore_c1x2<4, true, 8>(G, A, dir, s_c0, nc0, hot2s, nw, c1a, va, c1b, vb, A0, A0inv, cbuf,
                                             ccount, lane);
                    continue;
                }
                switch (G.r * 2u + (k == 16u ? 1u : 0u)) {
#define SD_RESTORE_CASE(RR)                                                                                       \
    case 2 * RR: restore_c1x2<RR, false, 0>(G, A, dir, s_c0, nc0, hot2s, nw, c1a, va, c1b, vb, A0, A0inv, cbuf,      \
                                           ccount, lane); break;                                                  \
    case 2 * RR + 1: restore_c1x2<RR, true, 0>(G, A, dir, s_c0, nc0, hot2s, nw, c1a, va, c1b, vb, A0, A0inv, cbuf,   \
                                              ccount, lane); break;
                    SD_RESTORE_CASE(3)
                    SD_RESTORE_CASE(4)
                    SD_RESTORE_CASE(5)
                    SD_RESTORE_CASE(6)
                    SD_RESTORE_CASE(7)
                    SD_RESTORE_CASE(8)
#undef SD_RESTORE_CASE
                    default: break;
                }
            }
            continue;
        }
        for (uint32_t m = 0; m < iters; m++) {
            const uint64_t j = jc * A.jchunk + (uint64_t)m * blockDim.x + threadIdx.x;
            const bool jvalid = j < J;
            const uint32_t i1 = (uint32_t)(j >> A.ulog);
            const uint32_t tt = (uint32_t)(j & ((1ull << A.ulog) - 1ull));
            const uint32_t c1 = jvalid ? he1[i1] : 0u;
            for (uint32_t q = 0; q < nc0; q++) {
                const uint32_t c0 = s_c0[q];  // same for the whole block
                const uint32_t L = c0 ^ c1;                 // BL(1): the low k bits of a
                const uint32_t Q = A0 * L;
                const uint32_t Qh = Q >> k, Ql = Q & kmask;
                bool found = jvalid;
                uint32_t u;
                if (k >= 16u) {
                    found = found && ((Ql >> (32u - k)) == (c0 & lowmask));
                    u = c0 >> lowbits;
                } else {
                    u = (c0 << (32u - 2u * k)) | tt;
                }
                const uint32_t H = (A0inv * ((u - Qh) & hmask)) & hmask;
                const uint32_t a = (H << k) | L;
                for (uint32_t i = 2; i < G.r && found; i++)
                    found = hot_at(hot2 + (uint64_t)(i - 2) * nw, dh_row(G, i, a, c0));
                const unsigned fb = __ballot_sync(0xFFFFFFFFu, found);
                if (!fb) continue;
                // append the candidates to the warp's buffer; flush 32 at a time
                if (found) cbuf[ccount + __popc(fb & ((1u << lane) - 1u))] = a;
                ccount += __popc(fb);
                __syncwarp();
                if (ccount >= 32) flush_cands(A, dir, cbuf, ccount, lane);
            }
        }
    }
    __syncwarp();
    flush_cands(A, dir, cbuf, ccount, lane);
}

// The tiles of direction 0 (tiles0 of them), then those of direction 1,
// dealt round-robin to the blocks of a 1-D grid.
__global__ void __launch_bounds__(256, 4)
k_restore(Geometry G, RestoreArgs A, uint64_t tiles0) {
    restore_body(G, A, 0, blockIdx.x, ~0ull, gridDim.x);
    if (G.dirs > 1) {
        const uint64_t first = ((uint64_t)blockIdx.x + gridDim.x - tiles0 % gridDim.x) % gridDim.x;
        restore_body(G, A, 1, first, ~0ull, gridDim.x);
    }
}

// k_estimate: SZ(a) = zero bits of ULE(a), the AND of a's r estimators, for
// every candidate in K (one warp per candidate, lanes over the estimator's
// words); keeps (a, SZ) when SZ <= szmax.  A direction whose K overflowed its
// capacity is skipped (it reports nothing).
// Candidates q_begin, q_begin + q_step, ... below q_end of direction `dir`,
// one warp each.
__device__ __forceinline__ void estimate_body(const Geometry &G, const RestoreArgs &A, uint32_t dir, uint64_t q_begin,
                                              uint64_t q_end, uint64_t q_step) {
    __shared__ unsigned long long s_hbuf[8][kWarpBuf];
    if (!(dir ? A.run[1] : A.run[0])) return;
    const unsigned long long nk = A.stats->ncand[dir];
    if (nk > A.cand_cap) return;
    const int szmax = dir ? A.szmax[1] : A.szmax[0];
    const uint32_t A0 = dir ? G.h[1].A0 : G.h[0].A0;
    const uint32_t lane = threadIdx.x & 31u;
    unsigned long long *hbuf = s_hbuf[threadIdx.x >> 5];
    uint32_t hcount = 0;
    const uint32_t *gdir = A.grid + (uint64_t)dir * G.dir_words;
    const uint32_t *cand = A.cand + (uint64_t)dir * A.cand_cap;
    const uint64_t q_stop = q_end < nk ? q_end : nk;
    if (G.wpc >= 4) {
        // lpc lanes per candidate, each ANDing 16-byte chunks of the r
        // estimators; the warp's 32 / lpc candidates are q, q + q_step, ...
        const uint32_t chunks = G.wpc >> 2;
        const uint32_t lpc = chunks < 32u ? chunks : 32u;
        const uint32_t cpw = 32u / lpc, sub = lane / lpc, sl = lane % lpc;
        const uint32_t kmask = (1u << G.k) - 1u;
        for (uint64_t q0 = q_begin; q0 < q_stop; q0 += (uint64_t)cpw * q_step) {
            const uint64_t q = q0 + (uint64_t)sub * q_step;
            const bool ok = q < q_stop;
            const uint32_t x = ok ? cand[q] : 0u;
            const uint32_t c0 = dh0(A0, G.k, x);
            uint32_t ones = 0;
            if (ok) {
                for (uint32_t c = sl; c < chunks; c += lpc) {
                    uint4 ule = make_uint4(~0u, ~0u, ~0u, ~0u);
#pragma unroll
                    for (uint32_t i = 0; i < 8; i++) {
                        if (i >= G.r) break;
                        const uint32_t ci = i == 0 ? c0 : ((shr_clamp(x, (i - 1u) * G.alpha) & kmask) ^ c0);
                        const uint4 v = __ldg(reinterpret_cast<const uint4 *>(gdir + (uint64_t)i * G.row_words +
                                                                              (uint64_t)ci * G.wpc) + c);
                        ule.x &= v.x; ule.y &= v.y; ule.z &= v.z; ule.w &= v.w;
                    }
                    ones += __popc(ule.x) + __popc(ule.y) + __popc(ule.z) + __popc(ule.w);
                }
            }
            for (uint32_t o = lpc >> 1; o > 0; o >>= 1) ones += __shfl_xor_sync(0xFFFFFFFFu, ones, o);
            const bool hit = ok && sl == 0 && (int)(G.g - ones) <= szmax;
            const unsigned hb = __ballot_sync(0xFFFFFFFFu, hit);
            if (!hb) continue;
            if (hit) hbuf[hcount + __popc(hb & ((1u << lane) - 1u))] = ((unsigned long long)x << 32) | (G.g - ones);
            hcount += __popc(hb);
            __syncwarp();
            if (hcount >= 32) flush_hits(A, dir, hbuf, hcount, lane);
        }
        __syncwarp();
        flush_hits(A, dir, hbuf, hcount, lane);
        return;
    }
    for (uint64_t q = q_begin; q < q_stop; q += q_step) {
        const uint32_t x = cand[q];
        const uint32_t c0 = dh0(A0, G.k, x);
        uint32_t ones = 0;
        for (uint32_t w = lane; w < G.wpc; w += 32) {
            uint32_t ule = 0xFFFFFFFFu;
            for (uint32_t i = 0; i < G.r; i++) {
                const uint32_t ci = (i == 0) ? c0 : dh_row(G, i, x, c0);
                ule &= __ldg(gdir + (uint64_t)i * G.row_words + (uint64_t)ci * G.wpc + w);
            }
            ones += __popc(ule);
        }
        ones = warp_sum(ones);
        const uint32_t SZ = G.g - ones;
        if ((int)SZ <= szmax) {
            if (lane == 0) hbuf[hcount] = ((unsigned long long)x << 32) | SZ;
            hcount++;
            __syncwarp();
            if (hcount >= 32) flush_hits(A, dir, hbuf, hcount, lane);
        }
    }
    __syncwarp();
    flush_hits(A, dir, hbuf, hcount, lane);
}

__global__ void __launch_bounds__(256)
k_estimate(Geometry G, RestoreArgs A) {
    const uint64_t nwarps = (uint64_t)gridDim.x * (blockDim.x >> 5);
    estimate_body(G, A, blockIdx.y, (uint64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5), ~0ull, nwarps);
}

// ------------------------------------------------------------------- sort
__device__ __forceinline__ void cswap(unsigned long long &a, unsigned long long &b, bool up) {
    if ((a > b) == up) {
        const unsigned long long t = a;
        a = b;
        b = t;
    }
}

// Bitonic sort of s[0, P) (P a power of two) by the whole block: each stage
// visits the P/2 compare-exchange pairs (i, i + j) directly.
__device__ __forceinline__ void bitonic_smem(unsigned long long *s, unsigned P) {
    for (unsigned kk = 2; kk <= P; kk <<= 1) {
        for (unsigned j = kk >> 1; j > 0; j >>= 1) {
            for (unsigned t = threadIdx.x; t < P / 2; t += blockDim.x) {
                const unsigned i = 2 * t - (t & (j - 1));  // low index of the t-th pair
                cswap(s[i], s[i + j], (i & kk) == 0);
            }
            __syncthreads();
        }
    }
}

// One block per direction: bitonic sort of up to kSortSmall hits in shared
// memory (padding with all-ones keys, which sort last).
__device__ __forceinline__ void sort_small_body(unsigned long long *hits, uint64_t hits_cap, StatBlock *st,
                                                uint32_t dir) {
    extern __shared__ unsigned long long s[];  // kSortSmall keys
    const unsigned long long n = st->nhits[dir];
    const unsigned long long nn = n < hits_cap ? n : hits_cap;
    if (nn > (unsigned long long)kSortSmall) {
        if (threadIdx.x == 0) st->big_sort[dir] = 1;
        return;
    }
    if (nn <= 1) return;
    unsigned P = 2;
    while (P < nn) P <<= 1;
    unsigned long long *hd = hits + (uint64_t)dir * hits_cap;
    for (unsigned i = threadIdx.x; i < P; i += blockDim.x) s[i] = i < nn ? hd[i] : ~0ull;
    __syncthreads();
    bitonic_smem(s, P);
    for (unsigned i = threadIdx.x; i < nn; i += blockDim.x) hd[i] = s[i];
}

__global__ void __launch_bounds__(1024)
k_sort_small(unsigned long long *hits, uint64_t hits_cap, StatBlock *st, uint2 run) {
    const uint32_t dir = blockIdx.x;
    if (!(dir ? run.y : run.x)) return;
    sort_small_body(hits, hits_cap, st, dir);
}

// Sort every segment keys[j*kSortSmall, (j+1)*kSortSmall) of keys[0, n) in
// shared memory (one block per segment, bitonic, padded with all-ones keys).
__global__ void __launch_bounds__(1024)
k_sort_segments(unsigned long long *keys, uint64_t n) {
    extern __shared__ unsigned long long s[];
    const uint64_t base = (uint64_t)blockIdx.x * kSortSmall;
    if (base >= n) return;
    const uint64_t left = n - base;
    const unsigned len = (unsigned)(left < (uint64_t)kSortSmall ? left : (uint64_t)kSortSmall);
    unsigned P = 1;
    while (P < len) P <<= 1;
    unsigned long long *kd = keys + base;
    for (unsigned i = threadIdx.x; i < P; i += blockDim.x) s[i] = i < len ? kd[i] : ~0ull;
    __syncthreads();
    bitonic_smem(s, P);
    for (unsigned i = threadIdx.x; i < len; i += blockDim.x) kd[i] = s[i];
}

// Merge neighbouring sorted runs of length L (the last may be shorter) from
// src into dst.  Keys are distinct, so an element's place in the merged run
// is its index in its own run plus the number of keys below it in the other
// run (a binary search): every element moves independently.
__global__ void k_merge_rank(const unsigned long long *__restrict__ src, unsigned long long *__restrict__ dst,
                             uint64_t n, uint64_t L) {
    const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
    for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride) {
        const uint64_t run = i / L;
        const uint64_t pb = (run & ~1ull) * L;
        const uint64_t a0 = pb, a1 = (pb + L < n) ? pb + L : n;
        const uint64_t b0 = a1, b1 = (pb + 2 * L < n) ? pb + 2 * L : n;
        const unsigned long long key = src[i];
        uint64_t lo, hi, own;
        if ((run & 1) == 0) {
            lo = b0; hi = b1; own = i - a0;
        } else {
            lo = a0; hi = a1; own = i - b0;
        }
        const uint64_t other0 = lo;
        while (lo < hi) {
            const uint64_t mid = lo + (hi - lo) / 2;
            if (src[mid] < key) lo = mid + 1;
            else hi = mid;
        }
        dst[pb + own + (lo - other0)] = key;
    }
}

// Merge all sorted segments of 2048 keys at once: a key's place in the
// output is its index in its own segment plus, for every other segment, the
// number of keys below it there (keys are distinct).  One launch instead of
// log2(segments) pairwise passes, for a few dozen segments at most.
constexpr uint32_t kMergeAllMaxSegs = 32;

__global__ void k_merge_all(const unsigned long long *__restrict__ src, unsigned long long *__restrict__ dst,
                            uint64_t n) {
    const uint32_t nseg = (uint32_t)((n + kSortSmall - 1) / kSortSmall);
    const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
    for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride) {
        const unsigned long long key = src[i];
        const uint32_t own = (uint32_t)(i / kSortSmall);
        uint64_t pos = i - (uint64_t)own * kSortSmall;
        for (uint32_t t = 0; t < nseg; t++) {
            if (t == own) continue;
            uint64_t lo = (uint64_t)t * kSortSmall;
            uint64_t hi = lo + kSortSmall < n ? lo + kSortSmall : n;
            const uint64_t base = lo;
            while (lo < hi) {
                const uint64_t mid = lo + (hi - lo) / 2;
                if (src[mid] < key) lo = mid + 1;
                else hi = mid;
            }
            pos += lo - base;
        }
        dst[pos] = key;
    }
}

// ----------------------------------------------------- sample sort (big)
// Hit lists longer than kSortSmall: nb buckets (a power of two, about 128
// keys each, up to 1024 buckets) split by nb - 1 splitters taken from a
// sorted sample of `over` keys per bucket (evenly spaced positions: 2 per
// bucket of 128, 8 for larger buckets); every key goes to the bucket of the
// splitters around it, and each bucket is sorted by one block in shared
// memory.  A bucket beyond kSortSmall keys (a sample that did not represent
// the keys) raises *overflow, and the host sorts the list again by the
// merge path.  Keys are distinct.

// bucket of `key`: the number of splitters below it
__device__ __forceinline__ uint32_t bucket_of(const unsigned long long *spl, uint32_t nb, unsigned long long key) {
    uint32_t lo = 0, hi = nb - 1;  // splitters spl[0 .. nb-2]
    while (lo < hi) {
        const uint32_t mid = (lo + hi) >> 1;
        if (spl[mid] < key) lo = mid + 1;
        else hi = mid;
    }
    return lo;
}

// One block: sort the sample, write the splitters, clear the counters.
__global__ void __launch_bounds__(1024)
k_ss_splitters(const unsigned long long *__restrict__ keys, uint64_t n, uint32_t nb, uint32_t over, SampleSortArgs S) {
    extern __shared__ unsigned long long smp[];  // nb * over keys
    const uint32_t m = nb * over;
    for (uint32_t i = threadIdx.x; i < m; i += blockDim.x) smp[i] = keys[((uint64_t)i * n) / m];
    for (uint32_t i = threadIdx.x; i <= nb; i += blockDim.x) {
        S.count[i] = 0;
        S.cursor[i] = 0;
    }
    if (threadIdx.x == 0) {
        S.ctl[0] = 0;  // count blocks done
        S.ctl[1] = 0;  // overflow
    }
    __syncthreads();
    if (m <= blockDim.x) {
        // a small sample: each thread places its key by counting the keys
        // below it (sample keys are distinct keys of the list)
        unsigned long long key = 0;
        uint32_t rank = 0;
        if (threadIdx.x < m) {
            key = smp[threadIdx.x];
            for (uint32_t j = 0; j < m; j++) rank += smp[j] < key;
        }
        __syncthreads();
        if (threadIdx.x < m) smp[rank] = key;
        __syncthreads();
    } else {
        bitonic_smem(smp, m);
    }
    for (uint32_t j = threadIdx.x; j + 1 < nb; j += blockDim.x) S.spl[j] = smp[(j + 1) * over - 1];
}

// Keys per bucket; the last block turns the counts into bucket offsets.
__global__ void __launch_bounds__(256)
k_ss_count(const unsigned long long *__restrict__ keys, uint64_t n, uint32_t nb, SampleSortArgs S) {
    __shared__ unsigned long long s_spl[kSampleMaxBuckets];
    __shared__ uint32_t s_hist[kSampleMaxBuckets];
    __shared__ bool s_last;
    for (uint32_t j = threadIdx.x; j < nb; j += blockDim.x) {
        if (j + 1 < nb) s_spl[j] = S.spl[j];
        s_hist[j] = 0;
    }
    __syncthreads();
    const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
    for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride)
        atomicAdd(&s_hist[bucket_of(s_spl, nb, keys[i])], 1u);
    __syncthreads();
    for (uint32_t j = threadIdx.x; j < nb; j += blockDim.x)
        if (s_hist[j]) atomicAdd(&S.count[j], s_hist[j]);
    __syncthreads();
    if (threadIdx.x == 0) {
        __threadfence();
        s_last = atomicAdd(&S.ctl[0], 1u) == gridDim.x - 1;
    }
    __syncthreads();
    if (!s_last) return;
    __threadfence();
    // exclusive scan of the nb <= 1024 counts, 4 consecutive ones per thread
    __shared__ uint32_t s_w[8];
    const uint32_t lane = threadIdx.x & 31u, wid = threadIdx.x >> 5;
    const uint32_t j0 = threadIdx.x * 4;
    uint32_t c[4], sum = 0;
#pragma unroll
    for (int q = 0; q < 4; q++) {
        c[q] = j0 + q < nb ? __ldcg(&S.count[j0 + q]) : 0u;
        sum += c[q];
    }
    uint32_t incl = sum;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const uint32_t v = __shfl_up_sync(0xFFFFFFFFu, incl, o);
        if ((int)lane >= o) incl += v;
    }
    if (lane == 31) s_w[wid] = incl;
    __syncthreads();
    uint32_t run = incl - sum;
    for (uint32_t w = 0; w < wid; w++) run += s_w[w];
#pragma unroll
    for (int q = 0; q < 4; q++) {
        if (j0 + q < nb) {
            S.off[j0 + q] = run;
            S.cursor[j0 + q] = run;
        }
        run += c[q];
    }
    if (j0 < nb && j0 + 4 >= nb) S.off[nb] = run;
}

// Every key to a free slot of its bucket in `out`: a block takes
// kScatterKeys keys per thread, ranks them per bucket in shared memory and
// reserves each bucket's run with one atomic.
constexpr uint32_t kScatterKeys = 4;
__global__ void __launch_bounds__(256)
k_ss_scatter(const unsigned long long *__restrict__ keys, unsigned long long *__restrict__ out, uint64_t n, uint32_t nb,
             SampleSortArgs S) {
    __shared__ unsigned long long s_spl[kSampleMaxBuckets];
    __shared__ uint32_t s_cnt[kSampleMaxBuckets];
    for (uint32_t j = threadIdx.x; j < nb; j += blockDim.x) {
        if (j + 1 < nb) s_spl[j] = S.spl[j];
        s_cnt[j] = 0;
    }
    __syncthreads();
    const uint64_t per_block = (uint64_t)blockDim.x * kScatterKeys;
    for (uint64_t base = (uint64_t)blockIdx.x * per_block; base < n; base += (uint64_t)gridDim.x * per_block) {
        unsigned long long key[kScatterKeys];
        uint32_t b[kScatterKeys], rank[kScatterKeys];
#pragma unroll
        for (uint32_t u = 0; u < kScatterKeys; u++) {
            const uint64_t i = base + (uint64_t)u * blockDim.x + threadIdx.x;
            b[u] = 0xFFFFFFFFu;
            if (i < n) {
                key[u] = keys[i];
                b[u] = bucket_of(s_spl, nb, key[u]);
                rank[u] = atomicAdd(&s_cnt[b[u]], 1u);
            }
        }
        __syncthreads();
        for (uint32_t j = threadIdx.x; j < nb; j += blockDim.x) {
            const uint32_t c = s_cnt[j];
            s_cnt[j] = c ? atomicAdd(&S.cursor[j], c) : 0u;  // the run's first slot
        }
        __syncthreads();
#pragma unroll
        for (uint32_t u = 0; u < kScatterKeys; u++)
            if (b[u] != 0xFFFFFFFFu) out[s_cnt[b[u]] + rank[u]] = key[u];
        __syncthreads();
        for (uint32_t j = threadIdx.x; j < nb; j += blockDim.x) s_cnt[j] = 0;
        __syncthreads();
    }
}

// One block per bucket: its keys of `in` sorted into the same places of
// `out` (up to 512 keys: each key placed by counting the keys below it;
// more: bitonic).
__global__ void __launch_bounds__(256)
k_ss_buckets(const unsigned long long *__restrict__ in, unsigned long long *__restrict__ out, SampleSortArgs S) {
    extern __shared__ unsigned long long s[];  // kSortSmall keys
    const uint32_t b = blockIdx.x;
    const uint32_t lo = S.off[b], len = S.off[b + 1] - lo;
    if (len > (uint32_t)kSortSmall) {
        if (threadIdx.x == 0) atomicOr(&S.ctl[1], 1u);
        return;
    }
    if (len == 0) return;
    if (len <= 512) {
        for (unsigned i = threadIdx.x; i < len; i += blockDim.x) s[i] = in[lo + i];
        __syncthreads();
        for (unsigned i = threadIdx.x; i < len; i += blockDim.x) {
            const unsigned long long key = s[i];
            uint32_t rank = 0;
            for (uint32_t j = 0; j < len; j++) rank += s[j] < key;
            out[lo + rank] = key;
        }
        return;
    }
    unsigned P = 1;
    while (P < len) P <<= 1;
    for (unsigned i = threadIdx.x; i < P; i += blockDim.x) s[i] = i < len ? in[lo + i] : ~0ull;
    __syncthreads();
    bitonic_smem(s, P);
    for (unsigned i = threadIdx.x; i < len; i += blockDim.x) out[lo + i] = s[i];
}

// ------------------------------------------------------------ reset/merge
__device__ __forceinline__ void reset_body(uint4 *grid4, uint64_t n4, StatBlock *st, uint32_t bx, uint32_t nbx) {
    const uint64_t stride = (uint64_t)nbx * blockDim.x;
    for (uint64_t i = (uint64_t)bx * blockDim.x + threadIdx.x; i < n4; i += stride)
        grid4[i] = make_uint4(0, 0, 0, 0);
    if (bx == 0) {
        uint32_t *w = reinterpret_cast<uint32_t *>(st);
        for (uint32_t i = threadIdx.x; i < sizeof(StatBlock) / 4; i += blockDim.x) w[i] = 0;
    }
}

__global__ void k_reset(uint4 *grid4, uint64_t n4, StatBlock *st) { reset_body(grid4, n4, st, blockIdx.x, gridDim.x); }

__global__ void k_merge_or(uint4 *dst, const uint4 *__restrict__ src, uint64_t n4) {
    const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
    for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n4; i += stride) {
        const uint4 a = dst[i], b = __ldg(src + i);
        dst[i] = make_uint4(a.x | b.x, a.y | b.y, a.z | b.z, a.w | b.w);
    }
}

// ------------------------------------------------------- batched closes
// The same kernels over an array of jobs, one grid dimension per job.
__global__ void __launch_bounds__(256) k_row_stats_many(const CloseJob *__restrict__ J) {
    const CloseJob &j = J[blockIdx.y];
    if (j.stats_done) return;  // the job's fold wrote its statistics
    row_stats_body(j.A.grid, j.G, j.zhot, const_cast<uint32_t *>(j.A.hotmap), j.A.stats, blockIdx.x, gridDim.x);
}

__global__ void __launch_bounds__(1024) k_compact_many(const CloseJob *__restrict__ J) {
    const CloseJob &j = J[blockIdx.y];
    compact_body(j.A.hotmap, j.G, const_cast<uint32_t *>(j.A.he), 2, blockIdx.x);
}

// Work of all (job, direction) segments laid end to end: segment s = 2 job +
// dir starts at base[s] (non-decreasing, base[2 count] = total).  The last
// segment whose start is at or below x holds item x.
__device__ __forceinline__ uint32_t segment_of(const unsigned long long *base, uint32_t nseg, uint64_t x) {
    uint32_t lo = 0, hi = nseg;  // base[lo] <= x < base[hi]
    while (hi - lo > 1) {
        const uint32_t mid = (lo + hi) >> 1;
        if (base[mid] <= x) lo = mid;
        else hi = mid;
    }
    return lo;
}

// Every block takes a contiguous run of the jobs' restore tiles (tile_base:
// host-computed tile offsets per segment), so that blocks share the work of
// the jobs in proportion to their tiles.
__global__ void __launch_bounds__(256, 4)
k_restore_many(const CloseJob *__restrict__ J, const unsigned long long *__restrict__ tile_base, uint32_t count) {
    const uint64_t total = tile_base[2 * count];
    const uint64_t per = (total + gridDim.x - 1) / gridDim.x;
    uint64_t a = (uint64_t)blockIdx.x * per;
    const uint64_t b = a + per < total ? a + per : total;
    while (a < b) {
        const uint32_t sg = segment_of(tile_base, 2 * count, a);
        const uint64_t end = tile_base[sg + 1] < b ? tile_base[sg + 1] : b;
        const CloseJob &j = J[sg >> 1];
        restore_body(j.G, j.A, sg & 1u, a - tile_base[sg], end - tile_base[sg], 1);
        a = end;
    }
}

// Candidate offsets per segment (0 for a direction that did not run or
// whose K overflowed its capacity), for the flat estimate below: one block,
// 1024 segments at a time, a block scan per batch of segments.
__global__ void __launch_bounds__(1024)
k_cand_base(const CloseJob *__restrict__ J, uint32_t count, unsigned long long *__restrict__ base) {
    __shared__ unsigned long long s_warp[32];
    __shared__ unsigned long long s_carry;
    const uint32_t lane = threadIdx.x & 31u, wid = threadIdx.x >> 5;
    if (threadIdx.x == 0) s_carry = 0;
    __syncthreads();
    for (uint32_t s0 = 0; s0 < 2 * count; s0 += blockDim.x) {
        const uint32_t sg = s0 + threadIdx.x;
        unsigned long long c = 0;
        if (sg < 2 * count) {
            const CloseJob &j = J[sg >> 1];
            const uint32_t d = sg & 1u;
            if (d < j.G.dirs && (d ? j.A.run[1] : j.A.run[0])) {
                const unsigned long long nk = j.A.stats->ncand[d];
                if (nk <= j.A.cand_cap) c = nk;
            }
        }
        unsigned long long incl = c;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const unsigned long long v = __shfl_up_sync(0xFFFFFFFFu, incl, o);
            if ((int)lane >= o) incl += v;
        }
        if (lane == 31) s_warp[wid] = incl;
        __syncthreads();
        if (wid == 0) {
            unsigned long long x = lane < (blockDim.x >> 5) ? s_warp[lane] : 0;
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const unsigned long long v = __shfl_up_sync(0xFFFFFFFFu, x, o);
                if ((int)lane >= o) x += v;
            }
            s_warp[lane] = x;  // inclusive over warps
        }
        __syncthreads();
        const unsigned long long carry = s_carry;
        const unsigned long long excl = carry + incl - c + (wid ? s_warp[wid - 1] : 0);
        if (sg < 2 * count) base[sg] = excl;
        __syncthreads();
        if (threadIdx.x == blockDim.x - 1) s_carry = carry + s_warp[(blockDim.x >> 5) - 1];
        __syncthreads();
    }
    if (threadIdx.x == 0) base[2 * count] = s_carry;
}

// Every warp takes a contiguous run of the jobs' candidates.
__global__ void __launch_bounds__(256)
k_estimate_many(const CloseJob *__restrict__ J, const unsigned long long *__restrict__ cand_base, uint32_t count) {
    const uint64_t total = cand_base[2 * count];
    const uint64_t nwarps = (uint64_t)gridDim.x * (blockDim.x >> 5);
    const uint64_t per = (total + nwarps - 1) / nwarps;
    uint64_t a = ((uint64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5)) * per;
    const uint64_t b = a + per < total ? a + per : total;
    while (a < b) {
        const uint32_t sg = segment_of(cand_base, 2 * count, a);
        const uint64_t end = cand_base[sg + 1] < b ? cand_base[sg + 1] : b;
        const CloseJob &j = J[sg >> 1];
        estimate_body(j.G, j.A, sg & 1u, a - cand_base[sg], end - cand_base[sg], 1);
        a = end;
    }
}

__global__ void __launch_bounds__(1024) k_sort_small_many(const CloseJob *__restrict__ J) {
    const CloseJob &j = J[blockIdx.y];
    const uint32_t dir = blockIdx.x;
    if (!(dir ? j.A.run[1] : j.A.run[0])) return;
    sort_small_body(j.A.hits, j.A.hits_cap, j.A.stats, dir);
}

// Every job's StatBlock, and the first min(hits, kSortSmall) hit keys of
// each direction, into contiguous buffers (one copy to the host for all).
__global__ void __launch_bounds__(256)
k_gather_many(const CloseJob *__restrict__ J, StatBlock *__restrict__ st_out, unsigned long long *__restrict__ hits_out) {
    const CloseJob &j = J[blockIdx.x];
    const uint32_t *src = reinterpret_cast<const uint32_t *>(j.A.stats);
    uint32_t *dst = reinterpret_cast<uint32_t *>(st_out + blockIdx.x);
    for (uint32_t i = threadIdx.x; i < sizeof(StatBlock) / 4; i += blockDim.x) dst[i] = src[i];
    for (uint32_t d = 0; d < j.G.dirs; d++) {
        if (!(d ? j.A.run[1] : j.A.run[0])) continue;
        const unsigned long long n = j.A.stats->nhits[d];
        uint64_t m = n < j.A.hits_cap ? n : j.A.hits_cap;
        if (m > (uint64_t)kSortSmall) m = kSortSmall;
        const unsigned long long *h = j.A.hits + (uint64_t)d * j.A.hits_cap;
        unsigned long long *o = hits_out + ((uint64_t)blockIdx.x * 2 + d) * kSortSmall;
        for (uint32_t i = threadIdx.x; i < m; i += blockDim.x) o[i] = h[i];
    }
}

__global__ void k_reset_many(const CloseJob *__restrict__ J, uint64_t n4) {
    const CloseJob &j = J[blockIdx.y];
    reset_body(reinterpret_cast<uint4 *>(const_cast<uint32_t *>(j.A.grid)), n4, j.A.stats, blockIdx.x, gridDim.x);
}

// ---------------------------------------------------------------- launchers
static unsigned grid_for(uint64_t items, unsigned threads, int num_sms, unsigned per_sm) {
    uint64_t b = (items + threads - 1) / threads;
    const uint64_t cap = (uint64_t)num_sms * per_sm;
    if (b > cap) b = cap;
    return (unsigned)(b ? b : 1);
}

cudaError_t launch_row_stats(const uint32_t *grid, const Geometry &G, int zhot, uint32_t *hotmap,
                             StatBlock *st, int num_sms, cudaStream_t s) {
    const uint64_t ncell = (uint64_t)G.dirs * G.r << G.k;
    k_row_stats<<<grid_for(ncell, 256, num_sms, 8), 256, 0, s>>>(grid, G, zhot, hotmap, st);
    return cudaGetLastError();
}

cudaError_t launch_compact(const uint32_t *hotmap, const Geometry &G, uint32_t *he, uint32_t rows,
                           cudaStream_t s) {
    k_compact<<<G.dirs * rows, 1024, 0, s>>>(hotmap, G, he, rows);
    return cudaGetLastError();
}

// Tile shape of k_restore for A's sizes: preimages per (c0, c1), (c1, t)
// items per tile, and c0 values per tile -- enough work per tile to amortise
// its set-up while still giving every resident block about one tile.
void prepare_restore(const Geometry &G, RestoreArgs &A, int num_sms, uint32_t tiles_per_block) {
    const unsigned threads = 256;
    A.ulog = (G.k >= 16u) ? 0u : (32u - 2u * G.k);
    A.jchunk = 2 * threads;  // two c1 values per thread and step
    uint64_t tests = 0;
    for (uint32_t d = 0; d < G.dirs; d++)
        if (A.run[d]) tests += (uint64_t)A.n0[d] * ((uint64_t)A.n1[d] << A.ulog);
    // c0 values per tile: about tiles_per_block tiles for each of the
    // (up to) 8 blocks per SM, so that the last wave of tiles is short
    const uint64_t per_block = tests / ((uint64_t)num_sms * 8 * threads * tiles_per_block) + 1;
    A.tile0 = (uint32_t)(per_block < kRestoreTileMax ? per_block : kRestoreTileMax);
    const size_t hot_bytes = (size_t)(G.r - 2) * ((1u << G.k) >> 5) * 4;
    A.smem_hot = hot_bytes <= (size_t)200 * 1024;
}

// k_restore tiles of direction d (the same count the kernel derives)
static uint64_t restore_tiles_dir(const Geometry &G, const RestoreArgs &A, uint32_t d) {
    if (d >= G.dirs || !A.run[d] || A.n0[d] == 0 || A.n1[d] == 0) return 0;
    const uint64_t t0 = (A.n0[d] + A.tile0 - 1) / A.tile0;
    const uint64_t nc = (((uint64_t)A.n1[d] << A.ulog) + A.jchunk - 1) / A.jchunk;
    return t0 * nc;
}

cudaError_t launch_restore(const Geometry &G, RestoreArgs A, int num_sms, cudaStream_t s) {
    const unsigned threads = 256;
    prepare_restore(G, A, num_sms, 4);
    const size_t hot_bytes = (size_t)(G.r - 2) * ((1u << G.k) >> 5) * 4;
    const size_t smem = A.smem_hot ? hot_bytes : 16;
    const uint64_t tiles0 = restore_tiles_dir(G, A, 0);
    const uint64_t total = tiles0 + restore_tiles_dir(G, A, 1);
    if (total == 0) return cudaSuccess;
    int per_sm = 0;
    cudaError_t e = prepare_launch(reinterpret_cast<const void *>(k_restore), (int)threads, smem, &per_sm);
    if (e != cudaSuccess) return e;
    uint64_t blocks = (uint64_t)num_sms * per_sm;
    if (total < blocks) blocks = total;
    k_restore<<<(unsigned)blocks, threads, smem, s>>>(G, A, tiles0);
    return cudaGetLastError();
}

cudaError_t launch_estimate(const Geometry &G, const RestoreArgs &A, int num_sms, cudaStream_t s) {
    dim3 grid((unsigned)num_sms * 4, G.dirs);
    k_estimate<<<grid, 256, 0, s>>>(G, A);
    return cudaGetLastError();
}

cudaError_t launch_sort_small(unsigned long long *hits, uint64_t hits_cap, StatBlock *st,
                              const uint32_t run[2], uint32_t dirs, cudaStream_t s) {
    const int smem = kSortSmall * (int)sizeof(unsigned long long);
    int per_sm = 0;
    cudaError_t e = prepare_launch(reinterpret_cast<const void *>(k_sort_small), 1024, smem, &per_sm);
    if (e != cudaSuccess) return e;
    k_sort_small<<<dirs, 1024, smem, s>>>(hits, hits_cap, st, make_uint2(run[0], run[1]));
    return cudaGetLastError();
}

cudaError_t launch_sort_big(unsigned long long *keys, unsigned long long *tmp, uint64_t n, void *scratch, int num_sms,
                            cudaStream_t s, unsigned long long **out, int *launches, uint32_t **overflow) {
    const int smem = kSortSmall * (int)sizeof(unsigned long long);
    int per_sm = 0;
    cudaError_t e;
    *overflow = nullptr;
    if (scratch && n <= kSampleMaxKeys) {
        uint32_t nb = 2;
        while ((uint64_t)nb * 128 < n && nb < kSampleMaxBuckets) nb <<= 1;
        const uint32_t over = (uint64_t)nb * 256 >= n ? 2u : 8u;
        SampleSortArgs S;
        S.spl = static_cast<unsigned long long *>(scratch);
        S.count = reinterpret_cast<uint32_t *>(S.spl + kSampleMaxBuckets);
        S.off = S.count + kSampleMaxBuckets + 1;
        S.cursor = S.off + kSampleMaxBuckets + 1;
        S.ctl = S.cursor + kSampleMaxBuckets + 1;
        const int ssmem = (int)(nb * over * sizeof(unsigned long long));
        if ((e = prepare_launch(reinterpret_cast<const void *>(k_ss_splitters), 1024, ssmem, &per_sm)) != cudaSuccess)
            return e;
        if ((e = prepare_launch(reinterpret_cast<const void *>(k_ss_buckets), 256, smem, &per_sm)) != cudaSuccess)
            return e;
        const unsigned blocks = grid_for(n, 256, num_sms, 4);
        k_ss_splitters<<<1, 1024, ssmem, s>>>(keys, n, nb, over, S);
        k_ss_count<<<blocks, 256, 0, s>>>(keys, n, nb, S);
        k_ss_scatter<<<grid_for(n, 256 * kScatterKeys, num_sms, 4), 256, 0, s>>>(keys, tmp, n, nb, S);
        k_ss_buckets<<<nb, 256, smem, s>>>(tmp, keys, S);
        *launches = 4;
        *out = keys;
        *overflow = S.ctl + 1;
        return cudaGetLastError();
    }
    e = prepare_launch(reinterpret_cast<const void *>(k_sort_segments), 1024, smem, &per_sm);
    if (e != cudaSuccess) return e;
    const uint64_t segs = (n + kSortSmall - 1) / kSortSmall;
    k_sort_segments<<<(unsigned)segs, 1024, smem, s>>>(keys, n);
    *launches = 1;
    if (segs <= kMergeAllMaxSegs) {
        k_merge_all<<<grid_for(n, 256, num_sms, 8), 256, 0, s>>>(keys, tmp, n);
        *launches = 2;
        *out = tmp;
        return cudaGetLastError();
    }
    unsigned long long *a = keys, *b = tmp;
    for (uint64_t L = kSortSmall; L < n; L <<= 1) {
        k_merge_rank<<<grid_for(n, 256, num_sms, 8), 256, 0, s>>>(a, b, n, L);
        ++*launches;
        unsigned long long *t = a;
        a = b;
        b = t;
    }
    *out = a;
    return cudaGetLastError();
}

cudaError_t launch_reset(uint32_t *grid, uint64_t words, StatBlock *st, int num_sms, cudaStream_t s) {
    const uint64_t n4 = words / 4;
    k_reset<<<grid_for(n4, 256, num_sms, 8), 256, 0, s>>>(reinterpret_cast<uint4 *>(grid), n4, st);
    return cudaGetLastError();
}

// Batched launchers: the grid's first dimension is shared by all jobs (each
// job strides over its own work with it), the job index is the last one.
cudaError_t launch_stats_many(const CloseJob *J, uint32_t count, const Geometry &G, int num_sms, cudaStream_t s) {
    const uint64_t ncell = (uint64_t)G.dirs * G.r << G.k;
    const unsigned per_job = std::max(1u, grid_for(ncell, 256, num_sms, 8) / std::max(1u, count / 4));
    k_row_stats_many<<<dim3(per_job, count), 256, 0, s>>>(J);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    k_compact_many<<<dim3(G.dirs * 2, count), 1024, 0, s>>>(J);
    return cudaGetLastError();
}

cudaError_t launch_restore_many(const CloseJob *J, const CloseJob *Jh, uint32_t count, unsigned long long *tile_base_d,
                                unsigned long long *tile_base_h, unsigned long long *cand_base_d, int num_sms,
                                cudaStream_t s, int *launches) {
    *launches = 0;
    const Geometry &G = Jh[0].G;
    const unsigned threads = 256;
    const size_t hot_bytes = (size_t)(G.r - 2) * ((1u << G.k) >> 5) * 4;
    const size_t smem = Jh[0].A.smem_hot ? hot_bytes : 16;
    unsigned long long acc = 0;
    bool any = false;
    for (uint32_t i = 0; i < count; i++) {
        any = any || Jh[i].A.run[0] || Jh[i].A.run[1];
        for (uint32_t d = 0; d < 2; d++) {
            tile_base_h[2 * i + d] = acc;
            if (d < G.dirs) acc += restore_tiles_dir(G, Jh[i].A, d);
        }
    }
    tile_base_h[2 * count] = acc;
    if (!any) return cudaSuccess;
    cudaError_t e = cudaMemcpyAsync(tile_base_d, tile_base_h, (2 * count + 1) * sizeof(unsigned long long),
                                    cudaMemcpyHostToDevice, s);
    if (e != cudaSuccess) return e;
    if (acc > 0) {
        int per_sm = 0;
        e = prepare_launch(reinterpret_cast<const void *>(k_restore_many), (int)threads, smem, &per_sm);
        if (e != cudaSuccess) return e;
        const uint64_t blocks = std::min<uint64_t>((uint64_t)num_sms * per_sm, acc);
        k_restore_many<<<(unsigned)blocks, threads, smem, s>>>(J, tile_base_d, count);
        if ((e = cudaGetLastError()) != cudaSuccess) return e;
        ++*launches;
    }
    k_cand_base<<<1, 1024, 0, s>>>(J, count, cand_base_d);
    k_estimate_many<<<(unsigned)num_sms * 8, 256, 0, s>>>(J, cand_base_d, count);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    const int ssmem = kSortSmall * (int)sizeof(unsigned long long);
    int per_sm = 0;
    e = prepare_launch(reinterpret_cast<const void *>(k_sort_small_many), 1024, ssmem, &per_sm);
    if (e != cudaSuccess) return e;
    k_sort_small_many<<<dim3(G.dirs, count), 1024, ssmem, s>>>(J);
    *launches += 3;
    return cudaGetLastError();
}

cudaError_t launch_gather_many(const CloseJob *J, uint32_t count, StatBlock *st_out, unsigned long long *hits_out,
                               cudaStream_t s) {
    k_gather_many<<<count, 256, 0, s>>>(J, st_out, hits_out);
    return cudaGetLastError();
}

cudaError_t launch_reset_many(const CloseJob *J, uint32_t count, const Geometry &G, int num_sms, cudaStream_t s) {
    const uint64_t n4 = (uint64_t)G.dirs * G.dir_words / 4;
    const unsigned per_job = std::max(1u, grid_for(n4, 256, num_sms, 8) / std::max(1u, count / 4));
    k_reset_many<<<dim3(per_job, count), 256, 0, s>>>(J, n4);
    return cudaGetLastError();
}

cudaError_t launch_merge(uint32_t *dst, const uint32_t *src, uint64_t words, int num_sms, cudaStream_t s) {
    const uint64_t n4 = words / 4;
    k_merge_or<<<grid_for(n4, 256, num_sms, 8), 256, 0, s>>>(reinterpret_cast<uint4 *>(dst),
                                                            reinterpret_cast<const uint4 *>(src), n4);
    return cudaGetLastError();
}

}  // namespace sd
