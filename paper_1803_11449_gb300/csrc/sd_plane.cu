// sd_plane.cu -- Algorithm 1 (Update DHLA) binned by estimator bit: the
// default update of sd_update (tuning mode 6).
//
// For one pair and one direction, Algorithm 1 sets the SAME bit b = H1(elem)
// in each of the r estimators DH_i(key), i < r (Eq. 2): one hash H1 per pair
// and direction, shared by the rows (§3.2).  Call "plane (d, b)" bit b of
// every estimator of direction d: r rows of 2^k bits, one bit per estimator.
// All r bit-sets of a (pair, direction) fall in one plane, at positions that
// depend on the key alone.  So the update is binned by plane with ONE entry
// per pair and direction -- the key itself -- and the rows are hashed where
// the plane is held, in shared memory:
//
//   k_plane_bin    tiles of pairs: the keys sorted by plane in shared memory,
//                  each plane's run appended to its bin with coalesced
//                  stores (one reservation atomic per plane and tile).  The
//                  bins are laid out back to back (each starting on a
//                  16-byte boundary) from the previous round's counts plus
//                  slack; keys beyond a bin's capacity (traffic that shifted
//                  between rounds) set their bits directly with atomic ORs.
//                  The last block cuts each plane's bin into apply units.
//   k_plane_layout for a round of another size than the previous one (of
//                  enough pairs to go by): that round's per-plane counts
//                  scaled to this round's size, plus slack.
//   k_plane_count  for a round with no usable history (the first one, one
//                  over other directions, or one after a small round): the
//                  exact keys of every plane, and a layout without slack.
//   k_plane_apply  one unit (a plane and a range of its bin) per block step:
//                  the plane in shared memory, DH_0 and Eq. 2 of every key,
//                  r shared-memory ORs, then one bulk OR of the plane into
//                  the plane-major copy of the DHLA in L2
//                  (cp.reduce.async.bulk ... .or.b32, so units of one plane
//                  may run on several SMs).  The last block lays out the
//                  next round's bins from this round's counts.
//   k_plane_fold   (sd_fold.cu; window close, sd_get_grid, sd_merge) folds
//                  the plane-major copy into the estimator-major DHLA
//                  (grid |= planes^T) and clears it.
//
// Per pair this moves dirs keys (4 bytes each) through the bins instead of
// r * dirs bit positions, and the plane copy is swept once per round by
// the bulk reduction.  The result equals Algorithm 1's DHLA bit for bit: the
// effective DHLA of a handle is grid | planes^T at all times, and every step
// only ORs bits in.
//
// Plane-major layout: plane (d, b) is plane index d*g + b; its row i starts
// at word i * 2^k/32 and holds estimator c's bit at word c >> 5, bit c & 31;
// planes are ps words apart (r 2^k / 32 rounded up to 4 words).
#include "sd_common.cuh"

namespace sd {

namespace {

constexpr uint32_t kPlaneThreads = 512;   // k_plane_bin / k_plane_count block
constexpr uint32_t kApplyThreads = 512;   // k_plane_apply block (1024 where one plane fills the block's shared memory)
constexpr uint32_t kHeldReservations = 2;  // reservation results a thread holds across the scatter
constexpr uint32_t kBinTilesPerBlock = 8;   // k_plane_bin tiles per block (blocks retire as a round runs)
constexpr uint32_t kApplyUnitsPerBlock = 4; // k_plane_apply units per block

__device__ __forceinline__ uint32_t h1v(uint64_t A1, uint64_t B1, uint32_t lg, uint32_t y) {
    return (uint32_t)((A1 * (uint64_t)y + B1) >> (64u - lg));
}

// 16-byte load that stays in L2 for the next kernel of the round.
__device__ __forceinline__ uint4 ld_l2_v4(const uint4 *p) {
    uint4 v;
    asm("ld.global.cg.v4.u32 {%0,%1,%2,%3}, [%4];" : "=r"(v.x), "=r"(v.y), "=r"(v.z), "=r"(v.w) : "l"(p));
    return v;
}

// Block-wide exclusive scan of get(0..N) written through put(i, prefix);
// put(N, total) as well.  Each thread takes a contiguous chunk of indices.
// Ends with a barrier; s_warp holds 32 words of shared scratch.
template <typename Get, typename Put>
__device__ __forceinline__ void block_scan(uint32_t N, Get get, Put put, uint32_t *s_warp) {
    const uint32_t per = (N + blockDim.x - 1) / blockDim.x;
    const uint32_t i0 = min(threadIdx.x * per, N), i1 = min(i0 + per, N);
    uint32_t sum = 0;
    for (uint32_t i = i0; i < i1; i++) sum += get(i);
    const uint32_t lane = threadIdx.x & 31u, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
    uint32_t incl = sum;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const uint32_t v = __shfl_up_sync(0xFFFFFFFFu, incl, o);
        if ((int)lane >= o) incl += v;
    }
    __syncthreads();  // s_warp may still be read by an earlier scan
    if (lane == 31) s_warp[wid] = incl;
    __syncthreads();
    if (wid == 0) {
        uint32_t x = lane < nw ? s_warp[lane] : 0u;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const uint32_t v = __shfl_up_sync(0xFFFFFFFFu, x, o);
            if ((int)lane >= o) x += v;
        }
        if (lane < nw) s_warp[lane] = x;
    }
    __syncthreads();
    uint32_t run = incl - sum + (wid ? s_warp[wid - 1] : 0u);
    for (uint32_t i = i0; i < i1; i++) {
        const uint32_t v = get(i);
        put(i, run);
        run += v;
    }
    if (threadIdx.x == blockDim.x - 1) put(N, run);
    __syncthreads();
}

// Capacity of a bin for an expected count c: c plus an eighth and 32 slots
// of slack when `slack`, rounded up to 4 entries.
__device__ __forceinline__ uint32_t bin_cap(uint32_t c, bool slack) {
    return (c + (slack ? c / 8u + 32u : 0u) + 3u) & ~3u;
}

// One block: the bins of the next round from this round's per-plane counts
// (cnt, then kept in prev and cleared), bins back to back.  The caller has
// seen every count (last-block pattern).
__device__ __forceinline__ void write_layout(const PlaneArgs &P, bool slack, uint32_t *s_warp) {
    const uint32_t NB = P.nbins;
    auto cap_of = [&](uint32_t i) { return bin_cap(__ldcg(&P.cnt[i]), slack); };
    block_scan(NB, cap_of, [&](uint32_t i, uint32_t v) { P.binoff[i] = v; }, s_warp);
    for (uint32_t b = threadIdx.x; b < NB; b += blockDim.x) {
        const uint32_t c = __ldcg(&P.cnt[b]);
        P.cap[b] = bin_cap(c, slack);
        P.prev[b] = c;
        P.cnt[b] = 0;
    }
}

// The last block to call this (one call per block, counter at *done) gets
// true, after a fence that makes every earlier block's writes visible.
__device__ __forceinline__ bool last_block(uint32_t *done, bool *s_last) {
    __syncthreads();
    if (threadIdx.x == 0) {
        __threadfence();
        *s_last = atomicAdd(done, 1u) == gridDim.x - 1;
    }
    __syncthreads();
    if (!*s_last) return false;
    __threadfence();
    return true;
}

// Set the r bits of `key` in plane b of the plane-major copy directly (a
// key its bin had no room for).
template <int DIRS>
__device__ __forceinline__ void set_key_bits(const Geometry &G, const PlaneArgs &P, uint32_t b, uint32_t key) {
    const uint32_t A0 = (DIRS == 2 && (b >> G.lg)) ? G.h[1].A0 : G.h[0].A0;
    const uint32_t rw = (1u << G.k) >> 5;
    uint32_t *pl = P.planes + (uint64_t)b * P.ps;
    const uint32_t c0 = dh0(A0, G.k, key);
    red_or(pl + (c0 >> 5), 1u << (c0 & 31u));
    for (uint32_t i = 1; i < G.r; i++) {
        const uint32_t ci = dh_row(G, i, key, c0);
        red_or(pl + i * rw + (ci >> 5), 1u << (ci & 31u));
    }
}

}  // namespace

// ------------------------------------------------------------------ count
template <int DIRS>
__global__ void __launch_bounds__(kPlaneThreads)
k_plane_count(const uint32_t *__restrict__ pairs, uint64_t n, Geometry G, PlaneArgs P) {
    extern __shared__ uint32_t hist[];  // [nbins]
    __shared__ uint32_t s_warp[32];
    __shared__ bool s_last;
    const uint32_t NB = P.nbins, g = G.g, lg = G.lg;
    const uint64_t A1a = G.h[0].A1, B1a = G.h[0].B1, A1b = G.h[1].A1, B1b = G.h[1].B1;
    for (uint32_t b = threadIdx.x; b < NB; b += blockDim.x) hist[b] = 0;
    __syncthreads();
    auto count = [&](uint32_t s, uint32_t t) {
        atomicAdd(&hist[h1v(A1a, B1a, lg, t)], 1u);
        if (DIRS == 2) atomicAdd(&hist[g + h1v(A1b, B1b, lg, s)], 1u);
    };
    const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
    const uint64_t first = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (((uintptr_t)pairs & 15u) == 0) {
        // four 16-byte loads in flight per thread
        const uint4 *v4 = reinterpret_cast<const uint4 *>(pairs);
        const uint64_t n2 = n / 2;
        uint64_t u = first;
        for (; u + 3 * stride < n2; u += 4 * stride) {
            uint4 v[4];
#pragma unroll
            for (int j = 0; j < 4; j++) v[j] = ld_l2_v4(v4 + u + j * stride);
#pragma unroll
            for (int j = 0; j < 4; j++) {
                count(v[j].x, v[j].y);
                count(v[j].z, v[j].w);
            }
        }
        for (; u < n2; u += stride) {
            const uint4 v = ld_l2_v4(v4 + u);
            count(v.x, v.y);
            count(v.z, v.w);
        }
        if ((n & 1) && first == 0) count(pairs[2 * (n - 1)], pairs[2 * (n - 1) + 1]);
    } else {
        for (uint64_t p = first; p < n; p += stride) count(ld_stream_u32(pairs + 2 * p), ld_stream_u32(pairs + 2 * p + 1));
    }
    __syncthreads();
    for (uint32_t b = threadIdx.x; b < NB; b += blockDim.x)
        if (hist[b]) atomicAdd(&P.cnt[b], hist[b]);
    if (!last_block(&P.ctl[0], &s_last)) return;
    // every count is in cnt: bins of exactly this round's sizes
    write_layout(P, false, s_warp);
    if (threadIdx.x == 0) P.ctl[0] = 0;
}

// ----------------------------------------------------------------- layout
// One block: bins for a round of `num` pairs from the per-plane counts of a
// previous round of `den` pairs (prev), each count scaled by num / den
// (rounded up) and given slack.  Their total stays within the bins of a
// round of num pairs: sum ceil(prev num / den) <= keys + nbins.
__global__ void __launch_bounds__(1024) k_plane_layout(PlaneArgs P, uint64_t num, uint64_t den) {
    __shared__ uint32_t s_warp[32];
    auto cap_of = [&](uint32_t i) {
        return bin_cap((uint32_t)(((uint64_t)P.prev[i] * num + den - 1) / den), true);
    };
    block_scan(P.nbins, cap_of, [&](uint32_t i, uint32_t v) { P.binoff[i] = v; }, s_warp);
    for (uint32_t b = threadIdx.x; b < P.nbins; b += blockDim.x) P.cap[b] = cap_of(b);
}

// -------------------------------------------------------------------- bin
// A thread keeps PPT pairs' DIRS entries in registers as (key, plane << 16
// | rank) while the block counts them per plane; the tile is then scattered
// into plane order in shared memory as 64-bit (plane << 32 | key) entries
// and written out one thread per entry, so each plane's run goes to
// consecutive addresses of its bin.
template <int DIRS, int PPT, bool FULL>
__device__ __forceinline__ void bin_hash(uint32_t cnt, const uint32_t (&ps)[PPT], const uint32_t (&pt)[PPT],
                                         uint32_t g, uint32_t lg, uint64_t A1a, uint64_t B1a, uint64_t A1b,
                                         uint64_t B1b, uint32_t *hist, uint32_t (&key)[PPT * DIRS],
                                         uint32_t (&tag)[PPT * DIRS]) {
#pragma unroll
    for (int j = 0; j < PPT / 2; j++) {
        const uint32_t pu = threadIdx.x + (uint32_t)j * blockDim.x;  // 2-pair unit within the tile
#pragma unroll
        for (int q = 0; q < 2; q++) {
            const bool ok = FULL || 2 * pu + q < cnt;
#pragma unroll
            for (int d = 0; d < DIRS; d++) {
                const int e = (2 * j + q) * DIRS + d;
                key[e] = d ? pt[2 * j + q] : ps[2 * j + q];
                const uint32_t b = d ? g + h1v(A1b, B1b, lg, ps[2 * j + q]) : h1v(A1a, B1a, lg, pt[2 * j + q]);
                tag[e] = 0xFFFFFFFFu;
                if (ok) tag[e] = (b << 16) | atomicAdd(&hist[b], 1u);
            }
        }
    }
}

template <int DIRS, int PPT, int THREADS>
__global__ void __launch_bounds__(THREADS, 1024 / THREADS)
k_plane_bin(const uint32_t *__restrict__ pairs, uint64_t n, Geometry G, PlaneArgs P) {
    constexpr int E = PPT * DIRS;
    extern __shared__ unsigned long long sm64[];
    __shared__ uint32_t s_warp[32];
    __shared__ bool s_last;
    const uint32_t NB = P.nbins, g = G.g, lg = G.lg;
    const uint32_t TP = blockDim.x * PPT;
    unsigned long long *sent = sm64;                               // [DIRS TP] (plane << 32 | key), plane order
    uint2 *dst = reinterpret_cast<uint2 *>(sent + (size_t)DIRS * TP);  // [NB] (bin index of sorted position 0,
                                                                   //  sorted positions below .y fit the bin)
    uint32_t *hist = reinterpret_cast<uint32_t *>(dst + NB);       // [NB] entries of each plane in the tile
    uint32_t *offs = hist + NB;                                    // [NB] first sorted position of each plane
    const uint64_t A1a = G.h[0].A1, B1a = G.h[0].B1, A1b = G.h[1].A1, B1b = G.h[1].B1;
    const uint64_t ntiles = (n + TP - 1) / TP;
    const bool vec = ((uintptr_t)pairs & 15u) == 0;
    // planes owned by this thread in the scan (contiguous chunk)
    const uint32_t per = (NB + blockDim.x - 1) / blockDim.x;
    const uint32_t b0 = min(threadIdx.x * per, NB), b1 = min(b0 + per, NB);
    // this thread's pairs of tile t: 2-pair units threadIdx.x + j blockDim.x
    // (coalesced 16-byte loads where the buffer allows)
    auto load_tile = [&](uint64_t t, uint32_t (&ps)[PPT], uint32_t (&pt)[PPT]) {
        const uint64_t base = t * TP;
        const uint64_t left = t < ntiles ? n - base : 0;
        const uint32_t cnt = left < TP ? (uint32_t)left : TP;
#pragma unroll
        for (int j = 0; j < PPT / 2; j++) {
            const uint32_t pu = threadIdx.x + (uint32_t)j * blockDim.x;
            const uint64_t p = base + 2ull * pu;
            const bool ok0 = 2 * pu < cnt, ok1 = 2 * pu + 1 < cnt;
            ps[2 * j] = pt[2 * j] = ps[2 * j + 1] = pt[2 * j + 1] = 0u;
            if (vec && ok1) {
                const uint4 v = ld_stream_v4(reinterpret_cast<const uint4 *>(pairs + 2 * p));
                ps[2 * j] = v.x; pt[2 * j] = v.y; ps[2 * j + 1] = v.z; pt[2 * j + 1] = v.w;
            } else {
                if (ok0) { ps[2 * j] = ld_stream_u32(pairs + 2 * p); pt[2 * j] = ld_stream_u32(pairs + 2 * p + 1); }
                if (ok1) {
                    ps[2 * j + 1] = ld_stream_u32(pairs + 2 * p + 2);
                    pt[2 * j + 1] = ld_stream_u32(pairs + 2 * p + 3);
                }
            }
        }
    };
    for (uint32_t b = threadIdx.x; b < NB; b += blockDim.x) hist[b] = 0;
    __syncthreads();
    uint32_t nps[PPT], npt[PPT];  // the next tile's pairs, loaded while the current one is written out
    load_tile(blockIdx.x, nps, npt);
    for (uint64_t t = blockIdx.x; t < ntiles; t += gridDim.x) {
        const uint64_t left = n - t * TP;
        const uint32_t cnt = left < TP ? (uint32_t)left : TP;
        const bool full = cnt == TP;
        uint32_t key[E], tag[E];
        if (full) bin_hash<DIRS, PPT, true>(cnt, nps, npt, g, lg, A1a, B1a, A1b, B1b, hist, key, tag);
        else bin_hash<DIRS, PPT, false>(cnt, nps, npt, g, lg, A1a, B1a, A1b, B1b, hist, key, tag);
        __syncthreads();
        // planes of this thread's chunk: sorted offsets, and their runs
        // reserved in the bins (the first kHeldReservations atomics' results
        // are used after the scatter, so their round trip overlaps it; with
        // more planes per thread the rest are resolved at once)
        uint32_t run = 0;
        {
            uint32_t sum = 0;
            for (uint32_t b = b0; b < b1; b++) sum += hist[b];
            const uint32_t lane = threadIdx.x & 31u, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
            uint32_t incl = sum;
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const uint32_t v = __shfl_up_sync(0xFFFFFFFFu, incl, o);
                if ((int)lane >= o) incl += v;
            }
            if (lane == 31) s_warp[wid] = incl;
            __syncthreads();
            if (wid == 0) {
                uint32_t x = lane < nw ? s_warp[lane] : 0u;
#pragma unroll
                for (int o = 1; o < 32; o <<= 1) {
                    const uint32_t v = __shfl_up_sync(0xFFFFFFFFu, x, o);
                    if ((int)lane >= o) x += v;
                }
                if (lane < nw) s_warp[lane] = x;
            }
            __syncthreads();
            run = incl - sum + (wid ? s_warp[wid - 1] : 0u);
        }
        uint32_t res[kHeldReservations], rrun[kHeldReservations], rcap[kHeldReservations],
            roff[kHeldReservations];
#pragma unroll
        for (uint32_t q = 0; q < kHeldReservations; q++) {
            const uint32_t b = b0 + q;
            res[q] = 0;
            rrun[q] = run;
            rcap[q] = 0;
            roff[q] = 0;
            if (b < b1) {
                const uint32_t h = hist[b];
                offs[b] = run;
                if (h) {
                    res[q] = atomicAdd(&P.cnt[b], h);
                    rcap[q] = P.cap[b];
                    roff[q] = P.binoff[b];
                }
                hist[b] = 0;
                run += h;
            }
        }
        for (uint32_t b = b0 + kHeldReservations; b < b1; b++) {
            const uint32_t h = hist[b];
            offs[b] = run;
            if (h) {
                const uint32_t pos = atomicAdd(&P.cnt[b], h), c = P.cap[b];
                dst[b] = make_uint2(P.binoff[b] + pos - run, run + (c > pos ? c - pos : 0u));
            }
            hist[b] = 0;
            run += h;
        }
        __syncthreads();
        // scatter into plane order
#pragma unroll
        for (int e = 0; e < E; e++) {
            if (tag[e] == 0xFFFFFFFFu) continue;
            const uint32_t b = tag[e] >> 16;
            sent[offs[b] + (tag[e] & 0xFFFFu)] = ((unsigned long long)b << 32) | key[e];
        }
        load_tile(t + gridDim.x, nps, npt);
#pragma unroll
        for (uint32_t q = 0; q < kHeldReservations; q++) {
            const uint32_t b = b0 + q;
            if (b < b1)
                dst[b] = make_uint2(roff[q] + res[q] - rrun[q], rrun[q] + (rcap[q] > res[q] ? rcap[q] - res[q] : 0u));
        }
        __syncthreads();
        // write-out: sorted entry q of plane b goes to bins[dst[b].x + q]
        // while its bin has room (plain stores: a plane's run is a fraction
        // of a line, and the line is completed by other tiles; streaming
        // stores would push the partial lines to DRAM several times over)
        const uint32_t nent = cnt * DIRS;
#pragma unroll 4
        for (uint32_t q = threadIdx.x; q < nent; q += blockDim.x) {
            const unsigned long long ent = sent[q];
            const uint32_t b = (uint32_t)(ent >> 32);
            const uint2 d = dst[b];
            if (q < d.y) P.bins[(uint32_t)(d.x + q)] = (uint32_t)ent;
            else set_key_bits<DIRS>(G, P, b, (uint32_t)ent);
        }
    }
    // the last block: apply units of the bins' actual contents
    if (!last_block(&P.ctl[0], &s_last)) return;
    const uint32_t U = P.unit;
    block_scan(NB, [&](uint32_t i) { return (min(__ldcg(&P.cnt[i]), P.cap[i]) + U - 1u) / U; },
               [&](uint32_t i, uint32_t v) { P.unit_start[i] = v; }, s_warp);
    if (threadIdx.x == 0) {
        P.ctl[0] = 0;
        P.ctl[1] = 0;
        P.ctl[2] = 0;
    }
}

// ------------------------------------------------------------------ apply
template <int R>
__device__ __forceinline__ void apply_key(uint32_t *pl, const Geometry &G, uint32_t A0, uint32_t rw, uint32_t key) {
    const uint32_t c0 = dh0(A0, G.k, key);
    atomicOr(&pl[c0 >> 5], 1u << (c0 & 31u));
#pragma unroll
    for (int i = 1; i < R; i++) {
        const uint32_t ci = dh_row(G, (uint32_t)i, key, c0);
        atomicOr(&pl[(uint32_t)i * rw + (ci >> 5)], 1u << (ci & 31u));
    }
}

// With two plane buffers (nbuf = 2, where two planes fit the block's shared
// memory) a unit is applied in one buffer while the bulk reduction of the
// previous unit still reads the other; before a buffer is reused, its
// reduction must have finished reading it (wait_group.read allows one
// reduction, the other buffer's, to stay in flight).  Planes too large for
// two buffers leave one block per SM, which then runs 1024 threads.
template <int R, int THREADS>
__global__ void __launch_bounds__(THREADS)
k_plane_apply(Geometry G, PlaneArgs P, uint32_t nbuf, uint32_t per_block) {
    extern __shared__ uint4 pl4_all[];  // nbuf planes of ps words
    __shared__ uint32_t s_unit;
    __shared__ uint32_t s_warp[32];
    __shared__ bool s_last;
    const uint32_t NB = P.nbins;
    const uint32_t rw = (1u << G.k) >> 5;
    const uint32_t total = P.unit_start[NB];
    // a block takes at most per_block units (the grid holds enough blocks
    // for every unit), so that blocks retire as the round proceeds and
    // other streams' work (a window close) gets SMs in between
    for (uint32_t it = 0; it < per_block; it++) {
        uint4 *pl4 = pl4_all + (size_t)(it % nbuf) * (P.ps / 4);
        uint32_t *pl = reinterpret_cast<uint32_t *>(pl4);
        if (threadIdx.x == 0) {
            if (nbuf == 2) asm volatile("cp.async.bulk.wait_group.read 1;" ::: "memory");
            else asm volatile("cp.async.bulk.wait_group.read 0;" ::: "memory");
            s_unit = atomicAdd(&P.ctl[1], 1u);
        }
        __syncthreads();  // this buffer is free again; the unit is known
        const uint32_t x = s_unit;
        if (x >= total) break;
        uint32_t lo = 0, hi = NB;  // the plane b with unit_start[b] <= x < unit_start[b + 1]
        while (hi - lo > 1) {
            const uint32_t mid = (lo + hi) >> 1;
            if (P.unit_start[mid] <= x) lo = mid;
            else hi = mid;
        }
        const uint32_t b = lo;
        const uint32_t beg = P.binoff[b] + (x - P.unit_start[b]) * P.unit;
        const uint32_t stop = P.binoff[b] + min(P.cnt[b], P.cap[b]);
        const uint32_t end = stop - beg < P.unit ? stop : beg + P.unit;
        const uint32_t A0 = (b >> G.lg) ? G.h[1].A0 : G.h[0].A0;
        for (uint32_t i = threadIdx.x; i < P.ps / 4; i += blockDim.x) pl4[i] = make_uint4(0, 0, 0, 0);
        __syncthreads();
        const uint4 *e4 = reinterpret_cast<const uint4 *>(P.bins + beg);  // beg is a multiple of 4
        const uint32_t n4 = (end - beg) / 4;
        uint32_t q = threadIdx.x;
        for (; q + 3 * blockDim.x < n4; q += 4 * blockDim.x) {
            uint4 v[4];
#pragma unroll
            for (int j = 0; j < 4; j++) v[j] = ld_stream_v4(e4 + q + j * blockDim.x);
#pragma unroll
            for (int j = 0; j < 4; j++) {
                apply_key<R>(pl, G, A0, rw, v[j].x); apply_key<R>(pl, G, A0, rw, v[j].y);
                apply_key<R>(pl, G, A0, rw, v[j].z); apply_key<R>(pl, G, A0, rw, v[j].w);
            }
        }
        for (; q < n4; q += blockDim.x) {
            const uint4 a = ld_stream_v4(e4 + q);
            apply_key<R>(pl, G, A0, rw, a.x); apply_key<R>(pl, G, A0, rw, a.y);
            apply_key<R>(pl, G, A0, rw, a.z); apply_key<R>(pl, G, A0, rw, a.w);
        }
        for (uint32_t r = beg + 4 * n4 + threadIdx.x; r < end; r += blockDim.x)
            apply_key<R>(pl, G, A0, rw, ld_stream_u32(P.bins + r));
        __syncthreads();
        if (threadIdx.x == 0) {
            // the plane's bits into the plane-major DHLA copy, ORed in L2
            asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
            asm volatile("cp.reduce.async.bulk.global.shared::cta.bulk_group.or.b32 [%0], [%1], %2;"
                         ::"l"(P.planes + (uint64_t)b * P.ps), "r"((uint32_t)__cvta_generic_to_shared(pl)),
                         "r"(P.ps * 4u)
                         : "memory");
            asm volatile("cp.async.bulk.commit_group;" ::: "memory");
        }
    }
    if (threadIdx.x == 0) asm volatile("cp.async.bulk.wait_group 0;" ::: "memory");
    // the last block: the next round's bins from this round's counts
    if (!last_block(&P.ctl[2], &s_last)) return;
    write_layout(P, true, s_warp);
}

// --------------------------------------------------------------- launchers
size_t plane_bin_smem_bytes(uint32_t tile_pairs, uint32_t dirs, uint32_t nbins) {
    return (size_t)dirs * tile_pairs * 8 + (size_t)nbins * 16;
}

template <int DIRS, int PPT, int THREADS>
static cudaError_t launch_plane_bin(const uint32_t *pairs, uint64_t n, const Geometry &G, const PlaneArgs &P,
                                    int num_sms, cudaStream_t s) {
    auto kern = k_plane_bin<DIRS, PPT, THREADS>;
    const size_t smem = plane_bin_smem_bytes(P.tile_pairs, DIRS, P.nbins);
    int per_sm = 0;
    cudaError_t e = prepare_launch(reinterpret_cast<const void *>(kern), THREADS, smem, &per_sm);
    if (e != cudaSuccess) return e;
    // about kBinTilesPerBlock tiles per block (not one persistent block per
    // SM), so that blocks retire as the round proceeds and other streams'
    // work gets SMs in between
    const uint64_t tiles = (n + P.tile_pairs - 1) / P.tile_pairs;
    uint64_t blocks = (tiles + kBinTilesPerBlock - 1) / kBinTilesPerBlock;
    if (blocks < (uint64_t)num_sms * per_sm) blocks = (uint64_t)num_sms * per_sm;
    if (tiles < blocks) blocks = tiles;
    kern<<<(unsigned)blocks, THREADS, smem, s>>>(pairs, n, G, P);
    return cudaGetLastError();
}

// tiles of 1024 to 4096 pairs: 512 threads with 2, 4 or 8 pairs each;
// 8192: 1024 threads with 8 each (one block per SM)
template <int DIRS>
static cudaError_t launch_plane_bin_d(const uint32_t *pairs, uint64_t n, const Geometry &G, const PlaneArgs &P,
                                      int num_sms, cudaStream_t s) {
    switch (P.tile_pairs) {
        case 1024: return launch_plane_bin<DIRS, 2, 512>(pairs, n, G, P, num_sms, s);
        case 2048: return launch_plane_bin<DIRS, 4, 512>(pairs, n, G, P, num_sms, s);
        case 4096: return launch_plane_bin<DIRS, 8, 512>(pairs, n, G, P, num_sms, s);
        case 8192: return launch_plane_bin<DIRS, 8, 1024>(pairs, n, G, P, num_sms, s);
        default: return cudaErrorInvalidValue;
    }
}

template <int R>
static cudaError_t launch_plane_apply(const Geometry &G, const PlaneArgs &P, uint64_t n, int num_sms,
                                     cudaStream_t s) {
    const uint32_t nbuf = (size_t)P.ps * 8 <= (size_t)100 * 1024 ? 2u : 1u;
    auto kern = nbuf == 2 ? k_plane_apply<R, kApplyThreads> : k_plane_apply<R, 2 * kApplyThreads>;
    const uint32_t threads = nbuf == 2 ? kApplyThreads : 2 * kApplyThreads;
    const size_t smem = (size_t)P.ps * 4 * nbuf;
    int per_sm = 0;
    cudaError_t e = prepare_launch(reinterpret_cast<const void *>(kern), (int)threads, smem, &per_sm);
    if (e != cudaSuccess) return e;
    // units of the round: at most (keys + slack) / unit + one partial unit per plane
    const uint64_t keys = (uint64_t)(P.nbins / G.g) * n;
    const uint64_t most = (keys + keys / 8 + 40ull * P.nbins) / P.unit + P.nbins;
    const uint32_t per_block = kApplyUnitsPerBlock;
    uint64_t blocks = (most + per_block - 1) / per_block;
    if (blocks < (uint64_t)num_sms * per_sm) blocks = (uint64_t)num_sms * per_sm;
    if (blocks > 0x7FFFFFFFull) return cudaErrorInvalidValue;
    kern<<<(unsigned)blocks, threads, smem, s>>>(G, P, nbuf, per_block);
    return cudaGetLastError();
}

cudaError_t launch_plane_round(const uint32_t *pairs, uint64_t n, const Geometry &G, const PlaneArgs &P, int num_sms,
                               cudaStream_t s, PlaneLayout layout, uint64_t prev_pairs) {
    if (n == 0) return cudaSuccess;
    if (layout == kLayoutScale) {
        if (prev_pairs == 0) return cudaErrorInvalidValue;
        k_plane_layout<<<1, 1024, 0, s>>>(P, n, prev_pairs);
        cudaError_t e = cudaGetLastError();
        if (e != cudaSuccess) return e;
    } else if (layout == kLayoutCount) {
        auto kern = G.dirs == 2 ? k_plane_count<2> : k_plane_count<1>;
        const size_t smem = (size_t)P.nbins * 4;
        int per_sm = 0;
        cudaError_t e = prepare_launch(reinterpret_cast<const void *>(kern), (int)kPlaneThreads, smem, &per_sm);
        if (e != cudaSuccess) return e;
        uint64_t blocks = (uint64_t)num_sms * per_sm;
        const uint64_t need = (n / 2 + kPlaneThreads - 1) / kPlaneThreads;
        if (need < blocks) blocks = need ? need : 1;
        kern<<<(unsigned)blocks, kPlaneThreads, smem, s>>>(pairs, n, G, P);
        if ((e = cudaGetLastError()) != cudaSuccess) return e;
    }
    cudaError_t e = G.dirs == 2 ? launch_plane_bin_d<2>(pairs, n, G, P, num_sms, s)
                                : launch_plane_bin_d<1>(pairs, n, G, P, num_sms, s);
    if (e != cudaSuccess) return e;
    switch (G.r) {
        case 3: return launch_plane_apply<3>(G, P, n, num_sms, s);
        case 4: return launch_plane_apply<4>(G, P, n, num_sms, s);
        case 5: return launch_plane_apply<5>(G, P, n, num_sms, s);
        case 6: return launch_plane_apply<6>(G, P, n, num_sms, s);
        case 7: return launch_plane_apply<7>(G, P, n, num_sms, s);
        case 8: return launch_plane_apply<8>(G, P, n, num_sms, s);
        default: return cudaErrorInvalidValue;
    }
}


}  // namespace sd
