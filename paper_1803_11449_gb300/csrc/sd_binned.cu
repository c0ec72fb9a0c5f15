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
    uint32_t base;  // first word of the direction (the DHLA has < 2^32 words here)
};

__device__ __forceinline__ DirConst dir_const(const Geometry &G, uint32_t d) {
    DirConst c;
    c.A0 = d ? G.h[1].A0 : G.h[0].A0;
    c.A1 = d ? G.h[1].A1 : G.h[0].A1;
    c.B1 = d ? G.h[1].B1 : G.h[0].B1;
    c.base = d ? (uint32_t)G.dir_words : 0u;
    return c;
}

// k_bin: a block handles tiles of blockDim*PPT pairs; each thread keeps the
// DIRS*R bit-sets of its PPT pairs in registers while the block counts them
// per slice, scans the counts, reserves runs in the bins, and scatters the
// entries into slice order in shared memory.  The write-out then walks the
// sorted entries with one thread per entry, so each slice's run is written
// with consecutive addresses.  A sorted entry is slice << 20 | local, where
// local = (word mod 2^slice_log2) << 5 | bit (slice_log2 <= 15, at most 4096
// slices).
struct DirHash {
    uint32_t A0[2];
    uint64_t A1[2], B1[2];
};

template <int R, int DIRS, int PPT, bool FULL>
__device__ __forceinline__ void bin_hash(const Geometry &G, const DirHash &H, const uint32_t (&base5)[DIRS][R],
                                         uint32_t cshift, uint32_t kmask, uint32_t sl5, uint32_t slice0,
                                         const uint32_t (&src)[PPT], const uint32_t (&dst)[PPT],
                                         const bool (&ok)[PPT], uint32_t *hist,
                                         uint32_t (&ent)[PPT * DIRS * R], uint32_t (&met)[PPT * DIRS * R]) {
    const uint32_t lmask = (1u << sl5) - 1u;
#pragma unroll
    for (int j = 0; j < PPT; j++) {
#pragma unroll
        for (int d = 0; d < DIRS; d++) {
            const uint32_t A0 = H.A0[d];
            const uint64_t A1 = H.A1[d];
            const uint64_t B1 = H.B1[d];
            const uint32_t key = d ? dst[j] : src[j], elem = d ? src[j] : dst[j];
            const uint32_t b = (uint32_t)((A1 * (uint64_t)elem + B1) >> (64u - G.lg));
            const uint32_t c0 = dh0(A0, G.k, key);
#pragma unroll
            for (int i = 0; i < R; i++) {
                const uint32_t ci = (i == 0) ? c0 : ((shr_clamp(key, (i - 1) * G.alpha) & kmask) ^ c0);
                const uint32_t bitidx = base5[d][i] + (ci << cshift) + b;  // global bit index
                const uint32_t sloc = bitidx >> sl5;  // slice within the link
                const int u = (j * DIRS + d) * R + i;
                ent[u] = ((slice0 + sloc) << 20) | (bitidx & lmask);
                if (FULL || ok[j]) met[u] = atomicAdd(&hist[sloc], 1u);
            }
        }
    }
}

// k_bin: a block handles tiles of blockDim*PPT pairs; each thread keeps the
// DIRS*R bit-sets of its PPT pairs in registers while the block counts them
// per slice, scans the counts, reserves runs in the bins, and scatters the
// entries into slice order in shared memory.  The write-out then walks the
// sorted entries with one thread per entry, so each slice's run is written
// with consecutive addresses.  A sorted entry is slice << 20 | local, where
// local = (bit index within the slice) = (word mod 2^slice_log2) << 5 | bit
// (slice_log2 <= 15, at most 4096 slices, fewer than 2^32 DHLA bits).
// Where a tile's pairs come from: one link given by the kernel parameters,
// or a table of links (a batched update of many windows in one launch), each
// with its own pairs, DHLA, hash constants and first slice.
struct TileSrc {
    const uint32_t *pairs;
    uint64_t n;        // pairs of the link
    uint64_t tile;     // tile index within the link
    uint32_t *grid;
    uint32_t slice0;   // first slice of the link in this launch
    DirHash H;
};

// Where a tile's sorted entries of one slice go: sorted entry q is written
// to dst + q while q < lim (the rest of the slice's run did not fit its bin).
struct Slot {
    uint32_t *dst;
    uint32_t lim;
    uint32_t pad;
};

// Slice qg (q within the tile's link) got bin positions b0, b0+1, ... for
// its sorted entries run, run+1, ...: entry run + i goes to bins[qg][b0 + i]
// while b0 + i < cap.
__device__ __forceinline__ void set_slot(Slot *slot, const BinArgs &B, uint32_t qg, uint32_t q, uint32_t b0,
                                         uint32_t run) {
    Slot sq;
    sq.dst = B.bins + (uint64_t)qg * B.cap + b0 - run;
    sq.lim = b0 < B.cap ? run + (B.cap - b0) : run;
    sq.pad = 0;
    slot[q] = sq;
}

template <int R, int DIRS, int PPT>
__global__ void __launch_bounds__(512)
k_bin(const uint32_t *__restrict__ pairs, uint64_t n, uint32_t *__restrict__ grid, Geometry G, BinArgs B,
      uint32_t lwpc, const LinkDesc *__restrict__ links, uint32_t nlinks, uint64_t ntiles_all, uint32_t SL) {
    constexpr int UPT = PPT * DIRS * R;  // bit-sets per thread per tile
    extern __shared__ uint32_t sm[];
    // indexed by the slice within the tile's link: a tile only touches the
    // SL slices of its own link
    Slot *slot = reinterpret_cast<Slot *>(sm);           // [SL], 16-byte aligned
    uint32_t *sorted = reinterpret_cast<uint32_t *>(slot + SL);  // [blockDim * UPT]
    uint32_t *hist = sorted + blockDim.x * UPT;          // [SL]
    uint32_t *offs = hist + SL;                          // [SL]
    __shared__ uint32_t warp_tot[32];

    const uint32_t TP = blockDim.x * PPT;
    const uint64_t ntiles = links ? ntiles_all : (n + TP - 1) / TP;
    const uint32_t lane = threadIdx.x & 31u, wid = threadIdx.x >> 5, nwarps = blockDim.x >> 5;
    const uint32_t sl = B.slice_log2, sl5 = sl + 5;
    const uint32_t kmask = (1u << G.k) - 1u, cshift = lwpc + 5;
    // first bit of row i of direction d
    uint32_t base5[DIRS][R];
#pragma unroll
    for (int d = 0; d < DIRS; d++)
#pragma unroll
        for (int i = 0; i < R; i++)
            base5[d][i] = ((d ? (uint32_t)G.dir_words : 0u) + (uint32_t)i * (uint32_t)G.row_words) << 5;
    if (blockIdx.x == 0 && threadIdx.x == 0) *B.work = 0;  // k_apply's slice counter
    for (uint32_t q = threadIdx.x; q < SL; q += blockDim.x) hist[q] = 0;
    for (uint64_t t = blockIdx.x; t < ntiles; t += gridDim.x) {
        TileSrc ts;
        if (links) {
            uint32_t l = 0;
            while (l + 1 < nlinks && links[l + 1].tile_start <= t) l++;
            const LinkDesc &L = links[l];
            ts.pairs = L.pairs;
            ts.n = L.n;
            ts.tile = t - L.tile_start;
            ts.grid = L.grid;
            ts.slice0 = L.slice0;
            ts.H.A0[0] = L.A0[0]; ts.H.A0[1] = L.A0[1];
            ts.H.A1[0] = L.A1[0]; ts.H.A1[1] = L.A1[1];
            ts.H.B1[0] = L.B1[0]; ts.H.B1[1] = L.B1[1];
        } else {
            ts.pairs = pairs;
            ts.n = n;
            ts.tile = t;
            ts.grid = grid;
            ts.slice0 = 0;
            ts.H.A0[0] = G.h[0].A0; ts.H.A0[1] = G.h[1].A0;
            ts.H.A1[0] = G.h[0].A1; ts.H.A1[1] = G.h[1].A1;
            ts.H.B1[0] = G.h[0].B1; ts.H.B1[1] = G.h[1].B1;
        }
        const bool vec = ((uintptr_t)ts.pairs & 15u) == 0;  // 16-byte loads of 2 pairs
        const uint64_t p0 = ts.tile * TP + (uint64_t)threadIdx.x * PPT;
        const bool full = (ts.tile + 1) * TP <= ts.n;
        uint32_t src[PPT], dst[PPT];
        bool ok[PPT];
        if (full && vec) {
            if (PPT == 2) {
                const uint4 v = ld_stream_v4(reinterpret_cast<const uint4 *>(ts.pairs + 2 * p0));
                src[0] = v.x; dst[0] = v.y; src[PPT - 1] = v.z; dst[PPT - 1] = v.w;
            } else {
#pragma unroll
                for (int j = 0; j < PPT; j += 2) {
                    const uint4 v = ld_stream_v4(reinterpret_cast<const uint4 *>(ts.pairs + 2 * (p0 + j)));
                    src[j] = v.x; dst[j] = v.y; src[j + 1] = v.z; dst[j + 1] = v.w;
                }
            }
#pragma unroll
            for (int j = 0; j < PPT; j++) ok[j] = true;
        } else {
            // partial tile, or pairs only 4- or 8-byte aligned: 32-bit loads
#pragma unroll
            for (int j = 0; j < PPT; j++) {
                ok[j] = p0 + j < ts.n;
                src[j] = ok[j] ? ld_stream_u32(ts.pairs + 2 * (p0 + j)) : 0u;
                dst[j] = ok[j] ? ld_stream_u32(ts.pairs + 2 * (p0 + j) + 1) : 0u;
            }
        }
        __syncthreads();  // previous tile written out, hist zero again
        uint32_t ent[UPT], met[UPT];
        if (full)
            bin_hash<R, DIRS, PPT, true>(G, ts.H, base5, cshift, kmask, sl5, ts.slice0, src, dst, ok, hist, ent,
                                         met);
        else
            bin_hash<R, DIRS, PPT, false>(G, ts.H, base5, cshift, kmask, sl5, ts.slice0, src, dst, ok, hist, ent,
                                          met);
        __syncthreads();
        // reserve each slice's run in its bin and scan hist into offs.  With
        // at most two slices per thread the reservations are issued first and
        // their results used only after the scatter, so the atomics' round
        // trip to L2 overlaps the scatter.
        uint32_t rb0[2], rrun[2], ds0 = 0, ds1 = 0;
        bool early = false;
        {
            const uint32_t per = (SL + blockDim.x - 1) / blockDim.x;
            const uint32_t s0 = min(threadIdx.x * per, SL), s1 = min(s0 + per, SL);
            early = per <= 2;
            ds0 = s0;
            ds1 = s1;
            uint32_t cnt = 0;
            if (early) {
#pragma unroll
                for (int j = 0; j < 2; j++) {
                    const uint32_t q = s0 + j;
                    if (q < s1) cnt += hist[q];
                }
            } else {
                for (uint32_t q = s0; q < s1; q++) cnt += hist[q];
            }
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
            if (early) {
#pragma unroll
                for (int j = 0; j < 2; j++) {
                    const uint32_t q = s0 + j;
                    rrun[j] = run;
                    rb0[j] = 0;
                    if (q < s1) {
                        const uint32_t hq = hist[q];
                        offs[q] = run;
                        if (hq) rb0[j] = atomicAdd(&B.count[ts.slice0 + q], hq);
                        run += hq;
                    }
                }
            } else {
                for (uint32_t q = s0; q < s1; q++) {
                    const uint32_t hq = hist[q];
                    offs[q] = run;
                    if (hq) set_slot(slot, B, ts.slice0 + q, q, atomicAdd(&B.count[ts.slice0 + q], hq), run);
                    run += hq;
                }
            }
        }
        __syncthreads();
        // scatter into slice order
#pragma unroll
        for (int u = 0; u < UPT; u++)
            if (full || ok[u / (DIRS * R)]) sorted[offs[(ent[u] >> 20) - ts.slice0] + met[u]] = ent[u];
        if (early) {
#pragma unroll
            for (int j = 0; j < 2; j++) {
                const uint32_t q = ds0 + j;
                if (q < ds1 && hist[q]) set_slot(slot, B, ts.slice0 + q, q, rb0[j], rrun[j]);
            }
        }
        __syncthreads();
        // write-out, one thread per entry; full bins fall back to red.or
        const uint64_t left = ts.n - ts.tile * TP;
        const uint32_t nu = (uint32_t)(left < TP ? left : TP) * DIRS * R;
        for (uint32_t q = threadIdx.x; q < nu; q += blockDim.x) {
            const uint32_t e = sorted[q];
            const Slot sq = slot[(e >> 20) - ts.slice0];
            if (q < sq.lim) {
                __stcs(sq.dst + q, e);  // evict-first: keeps the bin counters and the DHLA in L2
            } else {
                const uint32_t w = (((e >> 20) - ts.slice0) << sl) | ((e & 0xFFFFFu) >> 5);
                red_or(ts.grid + w, 1u << (e & 31u));
            }
        }
        for (uint32_t q = threadIdx.x; q < SL; q += blockDim.x) hist[q] = 0;
    }
}

__global__ void __launch_bounds__(1024)
k_apply(uint32_t *__restrict__ grid, BinArgs B, const LinkDesc *__restrict__ links, uint32_t slices_per_link) {
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
        const uint4 *bin4 = reinterpret_cast<const uint4 *>(bin);
        const uint32_t n4 = cnt / 4;  // cap is a multiple of 4: 16-byte aligned rows
#define SD_APPLY1(e) atomicOr(&slice[((e) & 0xFFFFFu) >> 5], 1u << ((e) & 31u))
        uint32_t q = threadIdx.x;
        for (; q + 3 * blockDim.x < n4; q += 4 * blockDim.x) {
            uint4 v[4];
#pragma unroll
            for (int j = 0; j < 4; j++) v[j] = ld_stream_v4(bin4 + q + j * blockDim.x);
#pragma unroll
            for (int j = 0; j < 4; j++) {
                SD_APPLY1(v[j].x); SD_APPLY1(v[j].y); SD_APPLY1(v[j].z); SD_APPLY1(v[j].w);
            }
        }
        for (; q < n4; q += blockDim.x) {
            const uint4 a = ld_stream_v4(bin4 + q);
            SD_APPLY1(a.x); SD_APPLY1(a.y); SD_APPLY1(a.z); SD_APPLY1(a.w);
        }
        for (uint32_t r = 4 * n4 + threadIdx.x; r < cnt; r += blockDim.x) {
            const uint32_t e = ld_stream_u32(bin + r);
            SD_APPLY1(e);
        }
#undef SD_APPLY1
        __syncthreads();
        // OR the slice into its DHLA (this block is the slice's only writer)
        uint32_t *g = grid;
        uint32_t local = s;
        if (links) {
            const uint32_t l = s / slices_per_link;
            local = s - l * slices_per_link;
            g = links[l].grid;
        }
        const uint64_t w0 = (uint64_t)local << B.slice_log2;
        const uint64_t left = B.total_words - w0;
        const uint32_t words = left < (uint64_t)SW ? (uint32_t)left : SW;
        uint4 *g4 = reinterpret_cast<uint4 *>(g + w0);
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

size_t bin_smem_bytes(uint32_t tile_pairs, uint32_t upd_per_pair, uint32_t S) {
    return (size_t)S * 16 + ((size_t)tile_pairs * upd_per_pair + 2ull * S) * 4;
}

template <int R, int DIRS, int PPT>
static cudaError_t launch_bin(const uint32_t *pairs, uint64_t n, uint32_t *grid, const Geometry &G,
                              const BinArgs &B, int num_sms, cudaStream_t s, const LinkDesc *links,
                              uint32_t nlinks, uint64_t ntiles_all, uint32_t slices_per_link) {
    auto kern = k_bin<R, DIRS, PPT>;
    const uint32_t threads = B.tile_pairs / PPT;
    const uint32_t SL = links ? slices_per_link : B.S;
    const size_t smem = bin_smem_bytes(B.tile_pairs, DIRS * R, SL);
    int per_sm = 0;
    cudaError_t e = prepare_launch(reinterpret_cast<const void *>(kern), (int)threads, smem, &per_sm);
    if (e != cudaSuccess) return e;
    const uint64_t tiles = links ? ntiles_all : (n + B.tile_pairs - 1) / B.tile_pairs;
    uint64_t blocks = (uint64_t)num_sms * (per_sm > 0 ? per_sm : 1);
    if (tiles < blocks) blocks = tiles ? tiles : 1;
    uint32_t lwpc = 0;
    while ((1u << lwpc) < G.wpc) lwpc++;
    kern<<<(unsigned)blocks, threads, smem, s>>>(pairs, n, grid, G, B, lwpc, links, nlinks, ntiles_all, SL);
    return cudaGetLastError();
}

template <int R>
static cudaError_t launch_bin_r(const uint32_t *pairs, uint64_t n, uint32_t *grid, const Geometry &G,
                                const BinArgs &B, int num_sms, cudaStream_t s, const LinkDesc *links,
                                uint32_t nlinks, uint64_t ntiles_all, uint32_t spl) {
    // 2 pairs per thread up to 1024-pair tiles (512 threads), else 4; the
    // API keeps tiles at 1024 pairs when dirs*r > 8 so registers suffice
    const bool two = B.tile_pairs <= 1024 || G.dirs * G.r > 8;
    if (G.dirs == 2) {
        if constexpr (2 * R <= 8) {
            if (!two) return launch_bin<R, 2, 4>(pairs, n, grid, G, B, num_sms, s, links, nlinks, ntiles_all, spl);
        }
        return launch_bin<R, 2, 2>(pairs, n, grid, G, B, num_sms, s, links, nlinks, ntiles_all, spl);
    }
    return two ? launch_bin<R, 1, 2>(pairs, n, grid, G, B, num_sms, s, links, nlinks, ntiles_all, spl)
               : launch_bin<R, 1, 4>(pairs, n, grid, G, B, num_sms, s, links, nlinks, ntiles_all, spl);
}

// One round: bin then apply (stream-ordered).  With `links` (a device table
// of nlinks links whose tiles number ntiles_all in total), pairs/n/grid are
// ignored and link l owns slices [l*slices_per_link, (l+1)*slices_per_link).
static cudaError_t launch_rounds(const uint32_t *pairs, uint64_t n, uint32_t *grid, const Geometry &G,
                                 const BinArgs &B, int num_sms, cudaStream_t s, const LinkDesc *links,
                                 uint32_t nlinks, uint64_t ntiles_all, uint32_t slices_per_link) {
    cudaError_t e;
    switch (G.r) {
        case 3: e = launch_bin_r<3>(pairs, n, grid, G, B, num_sms, s, links, nlinks, ntiles_all, slices_per_link); break;
        case 4: e = launch_bin_r<4>(pairs, n, grid, G, B, num_sms, s, links, nlinks, ntiles_all, slices_per_link); break;
        case 5: e = launch_bin_r<5>(pairs, n, grid, G, B, num_sms, s, links, nlinks, ntiles_all, slices_per_link); break;
        case 6: e = launch_bin_r<6>(pairs, n, grid, G, B, num_sms, s, links, nlinks, ntiles_all, slices_per_link); break;
        case 7: e = launch_bin_r<7>(pairs, n, grid, G, B, num_sms, s, links, nlinks, ntiles_all, slices_per_link); break;
        case 8: e = launch_bin_r<8>(pairs, n, grid, G, B, num_sms, s, links, nlinks, ntiles_all, slices_per_link); break;
        default: return cudaErrorInvalidValue;
    }
    if (e != cudaSuccess) return e;
    const size_t smem_apply = (size_t)4 << B.slice_log2;
    int per_sm_a = 0;
    e = prepare_launch(reinterpret_cast<const void *>(k_apply), 1024, smem_apply, &per_sm_a);
    if (e != cudaSuccess) return e;
    uint64_t ablocks = (uint64_t)num_sms * (per_sm_a > 0 ? per_sm_a : 1);
    if (B.S < ablocks) ablocks = B.S;
    k_apply<<<(unsigned)ablocks, 1024, smem_apply, s>>>(grid, B, links, slices_per_link);
    return cudaGetLastError();
}

cudaError_t launch_binned_chunk(const uint32_t *pairs, uint64_t n, uint32_t *grid, const Geometry &G,
                                const BinArgs &B, int num_sms, cudaStream_t s) {
    return launch_rounds(pairs, n, grid, G, B, num_sms, s, nullptr, 0, 0, B.S);
}

cudaError_t launch_binned_links(const LinkDesc *links_dev, uint32_t nlinks, uint64_t ntiles_all,
                                uint32_t slices_per_link, const Geometry &G, const BinArgs &B, int num_sms,
                                cudaStream_t s) {
    return launch_rounds(nullptr, 0, nullptr, G, B, num_sms, s, links_dev, nlinks, ntiles_all, slices_per_link);
}

}  // namespace sd
