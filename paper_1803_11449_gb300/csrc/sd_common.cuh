// sd_common.cuh -- types and device helpers shared by the library's
// translation units (update, close, C ABI).  Not part of the public ABI.
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

#include "sd.h"

namespace sd {

constexpr int kMaxRows = 8;

// Hash constants of one direction (see include/sd.h for the definitions).
struct HashDir {
    uint32_t A0;     // odd multiplier of DH_0
    uint32_t A0inv;  // its inverse mod 2^32 (restore)
    uint64_t A1;     // odd multiplier of H1
    uint64_t B1;     // additive constant of H1
};

// Shape of one handle's DHLA plus its hash constants, passed by value to
// every kernel.
struct Geometry {
    uint32_t g, r, k, alpha, dirs;
    uint32_t lg;          // log2 g
    uint32_t wpc;         // 32-bit words per estimator, g / 32
    uint64_t row_words;   // 2^k * wpc
    uint64_t dir_words;   // r * row_words
    HashDir h[2];
};

struct Tuning {
    uint32_t mode;           // 0 plain, 1 test-then-set, 2 test + warp de-dup,
                             // 3 filter + test, 4 filter + plain, 5 binned by
                             // DHLA slice, 6 binned by estimator bit (planes)
    uint32_t block_threads;
    uint32_t blocks_per_sm;
    uint32_t unroll;
    uint32_t filter_log2;    // log2 of the shared-memory filter entries (modes 3, 4)
    uint32_t bin_slice_log2; // mode 5: DHLA words per slice = 2^bin_slice_log2
    uint32_t bin_tile_pairs; // mode 5: pairs per binning tile
    uint32_t bin_chunk_log2; // mode 5: pairs per bin/apply round = 2^bin_chunk_log2
    uint32_t bin_slack_pct;  // mode 5: bin capacity over the mean fill, in percent
    uint32_t restore;        // 0 DH_0 inversion (k_restore), 1 staged join (sd_join.cu)
    uint32_t bin_batch_mib;  // mode 5, batched update: MiB of bins per round
    uint32_t plane_tile_pairs;  // mode 6: pairs per binning tile (1024, 2048 or 4096)
    uint32_t plane_round_log2;  // mode 6: pairs per count/bin/apply round, log2
    uint32_t plane_unit_log2;   // mode 6: bin entries per apply unit, log2
};

// The plane-binned update (sd_plane.cu): bins of keys per plane (d, b) =
// bit b of every estimator of direction d, and the plane-major DHLA copy.
// A round's bins are laid out from the previous round's counts (with slack)
// or, for a round without a usable history, from an exact count.
struct PlaneArgs {
    uint32_t *bins;        // the round's keys, plane by plane (each bin starts on 4 entries)
    uint32_t *cnt;         // [nbins] keys of each plane this round (zero between rounds)
    uint32_t *prev;        // [nbins] keys of each plane in the previous round
    uint32_t *binoff;      // [nbins + 1] first slot of each plane's bin
    uint32_t *cap;         // [nbins] slots of each plane's bin; keys beyond them are set directly
    uint32_t *unit_start;  // [nbins + 1] first apply unit of each plane
    uint32_t *ctl;         // [0] blocks done (count or bin), [1] apply units taken, [2] apply blocks done
    uint32_t *planes;      // [nbins][ps] plane-major DHLA copy
    uint32_t nbins;        // dirs * g
    uint32_t ps;           // words per plane: r 2^k / 32 rounded up to 4
    uint32_t unit;         // entries per apply unit (a multiple of 4)
    uint32_t tile_pairs;   // pairs per binning tile
};

// One link of a batched binned update (device memory table).
struct LinkDesc {
    const uint32_t *pairs;  // the link's pairs for this round
    uint64_t n;
    uint32_t *grid;         // the link's DHLA
    uint64_t tile_start;    // first tile of the link in the launch's tile order
    uint32_t slice0;        // first slice of the link in the launch's slice order
    uint32_t A0[2];
    uint64_t A1[2], B1[2];
};

struct BinArgs {
    uint32_t *bins;          // [S][cap]
    uint32_t *count;         // [S] entries appended this chunk (may exceed cap)
    uint32_t *work;          // apply's slice counter
    uint32_t S;              // slices
    uint32_t slice_log2;     // words per slice = 2^slice_log2
    uint32_t cap;            // entries per bin
    uint32_t tile_pairs;     // pairs per bin tile
    uint64_t total_words;    // dirs * dir_words
};


constexpr int kSortSmall = 2048;  // keys sorted by one block in shared memory
// Sample sort of hit lists beyond kSortSmall keys (up to kSampleMaxBuckets
// buckets of about 512 keys; longer lists take the merge path): splitters,
// per-bucket counts, offsets and cursors, and two control words (blocks
// done, overflow) in a scratch of kSampleScratchBytes per direction.
constexpr uint32_t kSampleMaxBuckets = 1024;
constexpr uint64_t kSampleMaxKeys = (uint64_t)kSampleMaxBuckets * 512;
constexpr size_t kSampleScratchBytes = 24 * 1024;
struct SampleSortArgs {
    unsigned long long *spl;  // [nb - 1] splitters, ascending
    uint32_t *count;          // [nb] keys per bucket
    uint32_t *off;            // [nb + 1] first slot of each bucket
    uint32_t *cursor;         // [nb] next free slot of each bucket
    uint32_t *ctl;            // [0] count blocks done, [1] a bucket overflowed
};

// Per-window counters, copied to the host in one transfer.
struct StatBlock {
    unsigned long long zr[2][kMaxRows];
    unsigned long long ncand[2];
    unsigned long long nhits[2];
    unsigned int nhot[2][kMaxRows];
    unsigned int big_sort[2];  // 1: hits did not fit the one-block sort
    unsigned int pad[2];
    unsigned long long jcount[2][kMaxRows];  // staged join: entries stage i produced
};

struct RestoreArgs {
    const uint32_t *grid;
    const uint32_t *he;      // [dirs][2][2^k]
    const uint32_t *hotmap;  // [dirs][r][2^k/32]
    uint32_t *cand;          // [dirs][cand_cap]
    unsigned long long *hits;  // [dirs][hits_cap]: (a << 32) | SZ
    StatBlock *stats;
    uint64_t cand_cap, hits_cap;
    uint32_t n0[2], n1[2];
    int32_t szmax[2];        // largest reported SZ; -1: none
    uint32_t run[2];
    uint32_t ulog;           // log2 of the preimage count per (c0, c1): max(0, 32-2k)
    uint32_t tile0;          // c0 values per block tile
    uint32_t jchunk;         // (c1, t) items per block tile
    int smem_hot;            // rows 2..r-1 of the hot bitmap staged in shared memory
};

// One window close of a batch (sd_close_many over handles of one DHLA
// shape): the handle's geometry (its hash constants), its restore arguments
// (all its device buffers: A.grid, A.he, A.hotmap, A.cand, A.hits, A.stats)
// and its hot threshold.  The batched close kernels take an array of these
// in device memory and pick the link from a grid dimension.
struct CloseJob {
    Geometry G;
    RestoreArgs A;
    int zhot;
    int stats_done;  // the fold already wrote the row statistics
};

// The staged join of sd_join.cu (the paper's Algorithms 3 and 4).
struct JoinArgs {
    const uint32_t *he;      // [dirs][r][2^k] hot lists
    unsigned long long *sub[2];  // [dirs][cap] intermediate buffers: (partial << 32) | c0
    uint64_t cap;
    uint32_t *cand;          // [dirs][cand_cap]
    uint64_t cand_cap;
    StatBlock *stats;        // ncand, jcount
    uint32_t n[2][kMaxRows]; // |HE(i)|
    uint32_t run[2];
};

// ---------------------------------------------------------------- hashes
// DH_0(x) = (A0 x mod 2^32) >> (32 - k)
__device__ __forceinline__ uint32_t dh0(uint32_t A0, uint32_t k, uint32_t x) {
    return (A0 * x) >> (32u - k);
}

// (x >> s) for s <= 31, 0 for s >= 32 (funnel shift with clamp).
__device__ __forceinline__ uint32_t shr_clamp(uint32_t x, uint32_t s) {
    return __funnelshift_rc(x, 0u, s);
}

// Eq. 2 for i >= 1, given DH_0(x) = c0.  The shift (i-1)*alpha is formed
// in registers (indexing a kernel-parameter array with a run-time row would
// copy the whole parameter block to local memory).
__device__ __forceinline__ uint32_t dh_row(const Geometry &G, uint32_t i, uint32_t x, uint32_t c0) {
    return (shr_clamp(x, (i - 1u) * G.alpha) & ((1u << G.k) - 1u)) ^ c0;
}

// H1(y) = (A1 y + B1 mod 2^64) >> (64 - log2 g)
__device__ __forceinline__ uint32_t h1(const HashDir &h, uint32_t lg, uint32_t y) {
    return (uint32_t)((h.A1 * (uint64_t)y + h.B1) >> (64u - lg));
}

// ------------------------------------------------------------ memory ops
// 16-byte streaming load of the pair stream: read once, do not keep in L1.
__device__ __forceinline__ uint4 ld_stream_v4(const uint4 *p) {
    uint4 v;
    asm("ld.global.nc.L1::no_allocate.v4.u32 {%0,%1,%2,%3}, [%4];"
                 : "=r"(v.x), "=r"(v.y), "=r"(v.z), "=r"(v.w)
                 : "l"(p));
    return v;
}

__device__ __forceinline__ uint32_t ld_stream_u32(const uint32_t *p) {
    uint32_t v;
    asm("ld.global.nc.L1::no_allocate.u32 %0, [%1];" : "=r"(v) : "l"(p));
    return v;
}

// Relaxed device-scope bitwise OR with no return value (a reduction).  Bits
// only ever go 0 -> 1 within a window, so no ordering is needed.
__device__ __forceinline__ void red_or(uint32_t *p, uint32_t v) {
    asm volatile("red.relaxed.gpu.global.or.b32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}

// Weak cached load of a DHLA word.  A stale 0 only costs a redundant OR; a
// stale 1 cannot happen because bits are never cleared inside a window.
__device__ __forceinline__ uint32_t ld_weak(const uint32_t *p) {
    uint32_t v;
    asm volatile("ld.global.u32 %0, [%1];" : "=r"(v) : "l"(p));
    return v;
}

// Launch set-up shared by every launcher: opts the kernel in to `smem` bytes
// of dynamic shared memory when above 48 KiB and returns its resident blocks
// per SM for (threads, smem).  Both are looked up once per (kernel, device,
// shape) and cached, so steady-state launches make no extra driver calls.
cudaError_t prepare_launch(const void *kernel, int threads, size_t smem, int *per_sm);

// ---------------------------------------------------------------- launchers
cudaError_t launch_update(const uint32_t *pairs, uint64_t n, uint32_t *grid, const Geometry &G,
                          const Tuning &T, int num_sms, cudaStream_t s);
cudaError_t launch_row_stats(const uint32_t *grid, const Geometry &G, int zhot, uint32_t *hotmap,
                             StatBlock *st, int num_sms, cudaStream_t s);
// HE(i) for rows 0..rows-1 of every direction, ascending: he[dir][row][2^k]
cudaError_t launch_compact(const uint32_t *hotmap, const Geometry &G, uint32_t *he, uint32_t rows, cudaStream_t s);
cudaError_t launch_restore(const Geometry &G, RestoreArgs A, int num_sms, cudaStream_t s);
cudaError_t launch_estimate(const Geometry &G, const RestoreArgs &A, int num_sms, cudaStream_t s);
// Host: DHLA layout and hash constants for a valid *p (as sd_create sets them).
void geometry_of(const sd_params *p, Geometry *out);

// Batched close over `count` jobs (device array J; Jh is the host copy,
// used for grid sizing): row stats + HE(0), HE(1) of every job; restore,
// estimate and small sorts; a gather of every job's StatBlock and first
// kSortSmall hits per direction into st_out[count] / hits_out[count][2]
// [kSortSmall]; the reset of every job's DHLA and counters.
cudaError_t launch_stats_many(const CloseJob *J, uint32_t count, const Geometry &G, int num_sms, cudaStream_t s);
void prepare_restore(const Geometry &G, RestoreArgs &A, int num_sms, uint32_t tiles_per_block);
// (restore and estimate spread all jobs' tiles / candidates over the whole
// grid: tile_base_* and cand_base_d hold 2 count + 1 offsets)
cudaError_t launch_restore_many(const CloseJob *J, const CloseJob *Jh, uint32_t count, unsigned long long *tile_base_d,
                                unsigned long long *tile_base_h, unsigned long long *cand_base_d, int num_sms,
                                cudaStream_t s, int *launches);
cudaError_t launch_gather_many(const CloseJob *J, uint32_t count, StatBlock *st_out, unsigned long long *hits_out,
                               cudaStream_t s);
cudaError_t launch_reset_many(const CloseJob *J, uint32_t count, const Geometry &G, int num_sms, cudaStream_t s);
// K by the staged join: r-2 launches (rows 2..r-1), both directions each
cudaError_t launch_join(const Geometry &G, const JoinArgs &J, int num_sms, cudaStream_t s);
cudaError_t launch_sort_small(unsigned long long *hits, uint64_t hits_cap, StatBlock *st,
                              const uint32_t run[2], uint32_t dirs, cudaStream_t s);
// Sort keys[0, n) ascending (distinct keys, n > kSortSmall) with tmp as
// scratch of the same size; *out gets the array holding the result.  With
// `scratch` (kSampleScratchBytes of device memory) and n <= kSampleMaxKeys
// the sample sort runs and *overflow points at a device word that is
// nonzero if it fell short (the caller then sorts again with scratch =
// nullptr: the merge path); otherwise *overflow is nullptr.
cudaError_t launch_sort_big(unsigned long long *keys, unsigned long long *tmp, uint64_t n, void *scratch, int num_sms,
                            cudaStream_t s, unsigned long long **out, int *launches, uint32_t **overflow);
cudaError_t launch_reset(uint32_t *grid, uint64_t words, StatBlock *st, int num_sms, cudaStream_t s);
cudaError_t launch_merge(uint32_t *dst, const uint32_t *src, uint64_t words, int num_sms, cudaStream_t s);
size_t bin_smem_bytes(uint32_t tile_pairs, uint32_t upd_per_pair, uint32_t S);
size_t plane_bin_smem_bytes(uint32_t tile_pairs, uint32_t dirs, uint32_t nbins);
// one round of the plane-binned update over n pairs: an exact count first
// when `count` (no usable layout from an earlier round), then bin and apply
// How a plane round gets its bin layout: the one the previous round left
// (its counts plus slack), that round's counts scaled by n / prev_pairs
// (plus slack), or an exact count of this round's keys.
enum PlaneLayout { kLayoutReuse = 0, kLayoutScale = 1, kLayoutCount = 2 };
cudaError_t launch_plane_round(const uint32_t *pairs, uint64_t n, const Geometry &G, const PlaneArgs &P, int num_sms,
                               cudaStream_t s, PlaneLayout layout, uint64_t prev_pairs);
// dst = OR of `count` arrays of `words` words at src (words a multiple of 4)
cudaError_t launch_or_words(uint32_t *dst, const uint32_t *src, uint64_t words, uint32_t count, int num_sms,
                            cudaStream_t s);
// key partition: counting pass (counts[parts] += ...) or scatter pass
// (cursor[parts] = each part's next slot; out gets (key, peer) pairs)
cudaError_t launch_partition(const uint32_t *pairs, uint64_t n, uint32_t dir, uint32_t parts,
                             unsigned long long *counts, unsigned long long *cursor, uint32_t *out, int num_sms,
                             cudaStream_t s, bool scatter);
// One handle's fold: grid |= planes^T (grid = planes^T where `clean`: the
// DHLA is all zero), planes = 0; with `st` (the window close, where
// fold_stats_fit), also the row statistics of k_row_stats: ZR and |HE(i)|
// added to st, every hot bitmap word written.
struct FoldJob {
    uint32_t *grid;
    uint32_t *planes;
    uint32_t clean;
    int zhot;
    StatBlock *st;       // nullptr: no statistics
    uint32_t *hotmap;    // [dirs][r][2^k/32]
};
// Whether a fold can compute the row statistics: tiles then hold every bit
// of their estimators (g/32 words of 8, 16 or 32).
inline bool fold_stats_fit(const Geometry &G) { return G.wpc >= 8 && G.wpc <= 32; }
// `one`'s fold, or (jobs != nullptr) the folds of njobs device-resident jobs
cudaError_t launch_plane_fold(const FoldJob &one, const FoldJob *jobs, uint32_t njobs, const Geometry &G, uint32_t ps,
                              int num_sms, cudaStream_t s);
cudaError_t launch_binned_chunk(const uint32_t *pairs, uint64_t n, uint32_t *grid, const Geometry &G,
                                const BinArgs &B, int num_sms, cudaStream_t s);
cudaError_t launch_binned_links(const LinkDesc *links_dev, uint32_t nlinks, uint64_t ntiles_all,
                                uint32_t slices_per_link, const Geometry &G, const BinArgs &B, int num_sms,
                                cudaStream_t s);

}  // namespace sd
