/*
 * sd.h -- C ABI of the GB300 library for network super-point detection with
 * the double-direction hash linear-estimator array (DHLA) of "Economical and
 * efficient network super points detection based on GPU" (arxiv 1803.11449).
 *
 * A handle owns one DHLA per traffic direction on one GPU: r rows ("LA"s) of
 * 2^k linear estimators of g bits each.  sd_update feeds (src, dst) IPv4
 * pairs into it (Algorithm 1); sd_close_window finds the hot estimators,
 * restores candidate super points by inverting the hash group, estimates
 * their cardinality (Eq. 4) and reports those at or above theta (Algorithm 2
 * and §4.2), then clears the DHLA for the next window.
 *
 * Conventions for every function:
 *   - Return 0 (SD_OK) on success and a negative SD_ERR_* code otherwise;
 *     sd_last_error(h) then holds a one-line message.
 *   - Nothing here takes ownership of caller memory.  Buffers the library
 *     returns (sd_report.hits) belong to the handle.
 *   - A handle is not thread-safe: calls on one handle must be serialised by
 *     the caller.  Different handles are independent.
 *   - All device work is ordered on the handle's CUDA stream
 *     (sd_params.cuda_stream, or a stream the handle creates), in call order.
 *     A window close runs its kernels on the handle's own side stream of the
 *     device's highest priority, joined to that stream before and after (so
 *     a close is scheduled ahead of other queued work, such as the next
 *     window's update of another handle).
 *
 * Hash group (a reading of §3.1/§3.2, which ask only for "random hash
 * functions"), fixed so every implementation agrees bit for bit:
 *   splitmix64 (Steele, Lea, Flood 2014) seeded with
 *   seed ^ (0x9E3779B97F4A7C15 * (dir + 1)) gives A0 (low 32 bits | 1),
 *   A1 (| 1) and B1, per direction dir.
 *   DH_0(x) = (A0 * x mod 2^32) >> (32 - k)                  (multiply-shift)
 *   DH_i(x) = ((x >> (i-1)*alpha) mod 2^k) xor DH_0(x)       (Eq. 2; shifts
 *             of 32 bits or more give 0)
 *   H1(y)   = (A1 * y + B1 mod 2^64) >> (64 - log2 g)        (multiply-add-shift)
 *   Direction 0 (outbound) keys on src and hashes dst; direction 1 (inbound)
 *   keys on dst and hashes src.
 */
#ifndef SD_H
#define SD_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define SD_OK 0
#define SD_ERR_ARG (-1)             /* invalid argument or parameter set */
#define SD_ERR_NOMEM (-2)           /* device or pinned host allocation failed */
#define SD_ERR_CUDA (-3)            /* a CUDA call failed; see sd_last_error */
#define SD_ERR_SATURATED (-4)       /* some row had ZR(i) = 0: psi = 1, Eq. 4 undefined */
#define SD_ERR_OVERLOAD (-5)        /* restore work or candidates over their caps */
#define SD_ERR_REPORT_OVERFLOW (-6) /* more hits than report_cap; count still exact */
#define SD_ERR_TOO_LARGE (-7)       /* sd_update_noalloc: the DHLA exceeds its fixed scratch */

/* Per-direction flags, in sd_report.flags at bit offset 8*dir. */
#define SD_FLAG_SATURATED 1u
#define SD_FLAG_OVERLOAD_PAIRS 2u  /* restore work bound over pair_cap: restore skipped */
#define SD_FLAG_OVERLOAD_CANDS 4u  /* |K| > cand_cap (or a staged-join list over its
                                      buffer): no hits; n_cand = cand_cap + 1 */
#define SD_FLAG_REPORT_OVERFLOW 8u /* hits beyond report_cap were dropped */

typedef struct sd_handle sd_handle;

/* Sketch and resource parameters.  A zero in a *_cap / stage field selects
 * its default. */
typedef struct {
    uint32_t g;           /* bits per linear estimator: power of two, 32..4096 */
    uint32_t r;           /* rows (LAs) per direction: 3..8 */
    uint32_t k;           /* 2^k estimators per row: 1..24 */
    uint32_t alpha;       /* bit-block stride of Eq. 2: 1 <= alpha <= k and
                             (r-2)*alpha + k >= 32 (the two restrictions of §3.3) */
    double theta;         /* super-point threshold (> 0) */
    uint64_t seed;        /* seed of the hash constants */
    uint32_t dirs;        /* 1: outbound (src keyed) only; 2: outbound and inbound */
    int32_t device;       /* CUDA device ordinal */
    uint64_t pair_cap;    /* restore work budget (the paper sets none): a direction's
                             restore is skipped (SD_FLAG_OVERLOAD_PAIRS) when
                             |HE(0)| * 2^(32-k), the number of keys whose DH_0 is a hot
                             estimator of row 0 (a superset of K), exceeds it; the
                             staged join (tuning restore = 1) is also skipped when its
                             first-stage tuples |HE(0)||HE(1)||HE(2)| exceed it;
                             default 2^32 */
    uint64_t cand_cap;    /* capacity for the candidate set K per direction;
                             default 2^20.  The restore stops once K has more members
                             (SD_FLAG_OVERLOAD_CANDS) */
    uint64_t report_cap;  /* most hits returned per close; default dirs*cand_cap */
    uint64_t stage_pairs; /* pairs per host-ingest chunk; default 2^22, or 2^24 when the
                             DHLA has more than 64 MiB */
    void *cuda_stream;    /* cudaStream_t for all device work, or NULL for a
                             handle-owned stream */
} sd_params;

/* One reported super point. */
typedef struct {
    uint32_t ip;       /* the host a0 */
    uint32_t sz;       /* SZ(a0): zero bits of ULE(a0), the AND of its r estimators */
    uint32_t dir;      /* 0 outbound (a0 was a src), 1 inbound (a0 was a dst) */
    uint32_t reserved;
    double est;        /* C(a0) of Eq. 4, computed in double on the host */
} sd_hit;

/* Result of one window.  Arrays are indexed [dir][row]; rows >= r and
 * directions >= dirs are zero. */
typedef struct {
    uint64_t n_pairs;       /* pairs fed to the window */
    uint64_t zr[2][8];      /* ZR(i): zero bits of row i (§3.3) */
    double psi[2];          /* psi of Lemma 1 with w' averaged over rows; -1 if saturated */
    uint32_t n_hot[2][8];   /* |HE(i)| */
    uint64_t n_cand[2];     /* |K| = #{a : DH_i(a) in HE(i) for all i}; cand_cap + 1 for a
                               direction flagged SD_FLAG_OVERLOAD_CANDS (|K| exceeds the
                               cap; the restore stopped there); 0 when the restore was
                               skipped */
    uint32_t zhot;          /* largest z_0 that is hot (z_0 < Zmin = g e^(-theta/g)) */
    uint32_t szmax[2];      /* largest SZ with C(SZ) >= theta (Eq. 4): hits have SZ <= szmax */
    uint32_t flags;         /* SD_FLAG_* at bit 8*dir */
    uint64_t n_hits_total;  /* hits found (exact even when truncated) */
    uint64_t n_hits;        /* hits returned in `hits` (<= report_cap) */
    const sd_hit *hits;     /* ordered by (dir, ip); owned by the handle, valid
                               until the next sd_close_window or sd_destroy */
} sd_report;

/* Update-kernel launch knobs, chosen by the autotuner.  Zero fields keep the
 * current value. */
typedef struct {
    uint32_t mode;          /* 0: one relaxed atomic OR per row;
                               1: test the bit first (Algorithm 1's test), skip set bits;
                               2: 1 + merge the targets of one word inside a warp;
                               3: a per-block shared-memory filter of bits known to
                                  be set, then 1;
                               4: the filter, then 0;
                               5: binned by DHLA slice: bit-sets sorted by slice through
                                  a scratch buffer, each slice updated in shared memory;
                               6: binned by estimator bit (the default where one bit
                                  plane, r 2^k bits, fits 192 KiB of shared memory): the
                                  keys of each direction sorted by H1(peer) -- the bit
                                  Algorithm 1 sets in all r estimators of the key -- then
                                  each bit plane's estimators DH_i(key) set in shared
                                  memory and ORed into a plane-major copy of the DHLA,
                                  folded into the DHLA before it is read */
    uint32_t block_threads; /* threads per block: 64..1024, multiple of 32 */
    uint32_t blocks_per_sm; /* resident blocks per SM the grid is sized for (0: as
                               many as fit) */
    uint32_t unroll;        /* 16-byte pair loads in flight per thread: 1, 2 or 4 */
    uint32_t filter_log2;   /* log2 of the filter's 8-byte entries: 8..14 */
    uint32_t bin_slice_log2; /* mode 5: DHLA words per slice, log2: 10..15 (raised
                                automatically to keep at most 4096 slices) */
    uint32_t bin_tile_pairs; /* mode 5: pairs per binning tile: a power of two, 64..2048
                                (64..1024 when dirs*r > 8) */
    uint32_t bin_chunk_log2; /* mode 5: pairs per bin-then-apply round, log2: 12..28 */
    uint32_t bin_slack_pct;  /* mode 5: bin capacity above the mean fill, percent
                                (0xFFFFFFFF sets 0); a full bin falls back to atomics */
    uint32_t restore;        /* how the close finds K (always set, like mode):
                                0: HE(0) x HE(1) joined, the rest of each address
                                   by inverting DH_0 (work |HE(0)||HE(1)| 2^max(0,32-2k));
                                1: the paper's staged join (§4.2, Algorithms 3-4):
                                   HE(0) x HE(1) x HE(2), then one row at a time
                                   through two intermediate buffers of 4 cand_cap
                                   entries per direction (allocated on first use);
                                   work |HE(0)||HE(1)||HE(2)| + the survivors x |HE(i)|;
                                   an intermediate list past its buffer flags the
                                   direction SD_FLAG_OVERLOAD_CANDS, and a first
                                   stage above pair_cap tuples SD_FLAG_OVERLOAD_PAIRS.
                                Both give the same K and the same report. */
    uint32_t bin_batch_mib;  /* sd_update_many driven by the handle: MiB of bins one
                                batched round may use (mode 5: bounds the links per
                                round; mode 6: bounds the lanes, bins of one plane
                                round each, at most 4); default 8192 */
    uint32_t plane_tile_pairs; /* mode 6: pairs per binning tile: 1024, 2048, 4096 or 8192
                                  (within 200 KiB of shared memory: 8 dirs bytes per pair
                                  plus 16 bytes per plane) */
    uint32_t plane_round_log2; /* mode 6: pairs per count/bin/apply round, log2: 10..28
                                  (also the members' rounds of a batch the handle drives) */
    uint32_t plane_unit_log2;  /* mode 6: bin entries per apply step, log2: 8..24 */
} sd_tuning;

/* Fill *p with the core-link configuration (g=512, r=4, k=16, alpha=8,
 * theta=1024, both directions, device 0) and default caps. */
int sd_default_params(sd_params *p);

/* Validate *p (§3.3 restrictions and layout limits); needs no GPU.
 * Returns SD_OK or SD_ERR_ARG. */
int sd_check_params(const sd_params *p);

/* Words of one direction's DHLA: r * 2^k * g/32.  Layout [row][estimator]
 * [g/32] uint32 words; bit b of an estimator is word b>>5, bit b&31.  0 if
 * *p is invalid. */
uint64_t sd_grid_words(const sd_params *p);

/* Device bytes a handle with *p holds once it has updated with its default
 * tuning: the DHLA, the hot sets, the candidate and hit buffers, and where
 * one bit plane fits (the default plane-binned update, tuning mode 6) the
 * plane-major DHLA copy and its counters (allocated on the first update);
 * 0 if *p is invalid.  Not counted, because they depend on the tuning or
 * the caller: the staging of host-pointer updates (2 * stage_pairs * 8
 * bytes) and the bins of the binned updates (sd_scratch_bytes). */
uint64_t sd_device_bytes(const sd_params *p);

/* Create a handle: allocate a zeroed DHLA per direction (the r LAs of 2^k
 * linear estimators of g bits each, §3.2, one per traffic direction of
 * §3.1) and the scratch of the close path (hot sets, K and the report of
 * Algorithm 2) on p->device.  *out is set only on success; on failure
 * nothing stays allocated and sd_last_error(NULL) says why. */
int sd_create(const sd_params *p, sd_handle **out);

/* Algorithm 1 over n pairs.  `pairs` holds n (src, dst) uint32 pairs,
 * interleaved (2n words), 4-byte aligned.  A device pointer is read in
 * place and the call returns once the work is queued: the buffer must stay
 * valid until the stream has executed it (sd_sync, or any later blocking
 * call on the handle).  A pinned host pointer is copied in chunks of
 * stage_pairs through the handle's device staging buffers, each chunk's
 * kernels overlapping the next chunk's copy.  A pageable host pointer is
 * read by the kernels in place when the device can access pageable memory
 * (cudaDevAttrPageableMemoryAccess, e.g. over a coherent CPU-GPU link), else
 * it is copied through pinned staging buffers as well.  For host pointers
 * the call returns once the caller's buffer may be reused.  n = 0 is a
 * no-op. */
int sd_update(sd_handle *h, const uint32_t *pairs, uint64_t n);

/* Close the window (Algorithm 2 with the §4.2 estimation step): per
 * direction compute z_0 and ZR(i), the hot sets HE(i), psi, the candidate
 * set K, SZ and C for each candidate, and report a0 when C(a0) >= theta.
 * Blocks until the report is ready, then clears the DHLA (asynchronously, in
 * stream order).  Returns SD_OK, or SD_ERR_SATURATED / SD_ERR_OVERLOAD /
 * SD_ERR_REPORT_OVERFLOW with *out still filled (flags say which direction);
 * the window is closed in every one of these cases. */
int sd_close_window(sd_handle *h, sd_report *out);

/* Close the windows of `count` handles at once: the same work and results
 * as sd_close_window on each, with the handles' GPU work overlapped across
 * their streams and one host synchronisation per close phase for all of
 * them (batched serving of many links).  outs[i] and rcs[i] receive handle
 * i's report and return code; the call returns SD_OK, or the first hard
 * error (SD_ERR_ARG / SD_ERR_NOMEM / SD_ERR_CUDA) among the rcs. */
int sd_close_many(sd_handle *const *hs, uint32_t count, sd_report *outs, int *rcs);

/* Algorithm 1 for `count` handles at once (batched windows of many links):
 * handle i gets the ns[i] pairs at pairs[i], exactly as sd_update would give
 * it.  Every link whose pairs are device-resident on hs[0]'s device and whose
 * DHLA has hs[0]'s shape (g, r, k, alpha, dirs) joins the batch, which runs
 * on hs[0]'s stream with hs[0]'s scratch (ordered after each member's
 * earlier work, and each member's later work after it); the other links
 * take sd_update.
 *   hs[0] in mode 6: each member in mode 6 runs its plane rounds (of up to
 *   2^plane_round_log2 pairs of hs[0]'s tuning, with its own tile and unit)
 *   through the bins of one of hs[0]'s lanes: hs[0]'s stream and up to three
 *   side streams of hs[0], each with bins of one round (as many lanes as
 *   bin_batch_mib holds); members go to lanes largest first, each to the
 *   lane with the fewest pairs so far, and a lane takes its members one
 *   after another.  Members in other modes take sd_update.
 *   hs[0] in mode 5: rounds take members round-robin, each contributing up
 *   to 2^bin_chunk_log2 pairs, as many as hs[0]'s bin_batch_mib of bins
 *   holds at the round's largest share (and at most 4096 slices in all),
 *   with one bin launch and one apply launch per round (binned by DHLA
 *   slice).
 * Returns the first error, if any. */
int sd_update_many(sd_handle *const *hs, const uint32_t *const *pairs, const uint64_t *ns, uint32_t count);

/* Device bytes of the binned update's bins that h allocates, with its
 * current tuning: mode 6, the bins of one plane round (of
 * 2^plane_round_log2 pairs) for its own rounds, times the lanes of a batch
 * of `links` members it drives (the plane copy is in sd_device_bytes); mode
 * 5, the slice bins of its own chunks (links <= 1) or of batched rounds
 * over `links` members (at most about bin_batch_mib MiB).  The bins grow to
 * the largest such need and are kept until sd_destroy.  0 when h does not
 * bin (tuning modes 0-4, or in mode 5 a DHLA of more than 4096 slices) or h
 * is NULL.  For memory budgets: a handle holds sd_device_bytes plus this. */
uint64_t sd_scratch_bytes(const sd_handle *h, uint32_t links);

/* Wait for all work queued on the handle's stream. */
int sd_sync(sd_handle *h);

/* Release every resource of the handle: its DHLAs (§3.2), the close
 * scratch of Algorithm 2 and any staging or binning scratch, after the work
 * queued on its stream has finished.  The report's hits become invalid.
 * NULL is a no-op. */
int sd_destroy(sd_handle *h);

/* Message of the last error on h (or of the last failed sd_create when h is
 * NULL).  Owned by the library. */
const char *sd_last_error(const sd_handle *h);

/* Copy direction dir's DHLA (sd_grid_words words) to / from host memory.
 * Used for checkpoints and parity checks; both block. */
int sd_get_grid(sd_handle *h, uint32_t dir, uint32_t *host_dst);
int sd_set_grid(sd_handle *h, uint32_t dir, const uint32_t *host_src);

/* After a close: row `row`'s hot bitmap of direction dir (2^k bits, packed
 * LSB-first into ceil(2^k/32) words) as of that close. */
int sd_get_hot(sd_handle *h, uint32_t dir, uint32_t row, uint32_t *host_bitmap);

/* After a close: copy up to `cap` members of direction dir's candidate set K
 * (unordered) into host_dst and return |K| (>= 0), or a negative error. */
int64_t sd_get_candidates(sd_handle *h, uint32_t dir, uint32_t *host_dst, uint64_t cap);

/* OR src's DHLAs into dst's (same g, r, k, alpha, seed, dirs and device).
 * This is the merge of local DHLAs from several monitors in §4.2, read as a
 * bitwise OR: the merged DHLA equals the one built from the union of the
 * streams.  Stream-ordered after the work already queued on both handles. */
int sd_merge(sd_handle *dst, sd_handle *src);

/* ------------------------------------------------------------------------
 * Several GPUs.  Two ways to spread a detection over GPUs follow from the
 * paper; the collectives themselves (NCCL or any other transport) are the
 * caller's, these calls are the device steps around them.
 *
 * Stream split, then merge (§4.2: the local DHLAs of several monitors or
 * GPUs merged into a global DHLA, read as a bitwise OR): each GPU runs
 * sd_update on its part of the window's stream; the DHLA images are
 * exported, ORed across GPUs (e.g. a reduce-scatter by all-to-all whose
 * parts sd_or_words combines, then an all-gather), ORed back into each
 * handle with sd_or_grid, and the window closed.  The merged DHLA equals
 * the DHLA of the whole stream, so the report is the one-GPU report.
 *
 * Key partition (§5: hosts divided by the low bits of their address): each
 * direction's pairs are grouped by key & (parts - 1) with
 * sd_partition_pairs, each group sent to the GPU that owns those keys
 * (e.g. an all-to-all), and fed there with sd_update_dir; each GPU's DHLA
 * holds its own keys only and nothing is merged.  A GPU's report is valid
 * for its own keys (hits of other keys are estimator collisions and are
 * dropped by the caller).
 * ------------------------------------------------------------------------ */

/* Algorithm 1 for direction `dir` alone: `pairs` holds n (key, peer) pairs
 * of that direction, interleaved -- (src, dst) for direction 0, (dst, src)
 * for direction 1 -- with the same memory rules as sd_update.  Used to feed
 * a key partition (each direction's keys arrive separately).  The window's
 * n_pairs counts the pairs given to sd_update and, of sd_update_dir, those
 * of direction 0. */
int sd_update_dir(sd_handle *h, uint32_t dir, const uint32_t *pairs, uint64_t n);

/* Copy h's DHLA, both directions in the sd_get_grid layout (dirs *
 * sd_grid_words words, direction 0 first), to `dst`: 16-byte aligned device
 * memory on h's device.  Stream-ordered on h's stream; returns once queued
 * (the image of the DHLA as of the work queued before it). */
int sd_export_grid(sd_handle *h, uint32_t *dst);

/* h's DHLA |= the image at `src` (layout as sd_export_grid; 16-byte aligned
 * device memory on h's device): the §4.2 merge of local DHLAs, read as a
 * bitwise OR, so the result is the DHLA of the union of the streams.
 * Stream-ordered on h's stream; `src` must stay valid until it has run. */
int sd_or_grid(sd_handle *h, const uint32_t *src);

/* dst[j] = src[j] | src[words + j] | ... | src[(count-1) words + j] for
 * j < words: the OR of `count` DHLA parts laid end to end (the reduction
 * step of an OR all-reduce; no collective library offers a bitwise-OR
 * reduction).  words must be a multiple of 4; dst and src are 16-byte
 * aligned device memory of the current device.  Runs on `cuda_stream`
 * (NULL: the legacy default stream); returns once queued. */
int sd_or_words(uint32_t *dst, const uint32_t *src, uint64_t words, uint32_t count, void *cuda_stream);

/* Group n (src, dst) pairs (device memory on h's device) by the key of
 * direction dir (src for 0, dst for 1): `out` (2n words, device memory)
 * receives (key, peer) pairs part by part, part q = key & (parts - 1) for
 * q = 0..parts-1 (within a part in no particular order), and counts[q]
 * (host) the pairs of part q.  parts is a power of two up to 1024.  Runs on
 * h's stream and blocks until `out` and counts are complete (the counts
 * size the caller's exchange).  §5's division of hosts by their low bits. */
int sd_partition_pairs(sd_handle *h, uint32_t dir, const uint32_t *pairs, uint64_t n, uint32_t parts,
                       uint32_t *out, uint64_t *counts);

/* Number of CUDA kernels the library has launched in this process, over all
 * handles (the init clear of sd_create included); for benchmarks that report
 * their launch count. */
uint64_t sd_kernel_launches(void);

/* Read or change the update-kernel launch knobs. */
int sd_get_tuning(const sd_handle *h, sd_tuning *out);
int sd_set_tuning(sd_handle *h, const sd_tuning *t);

/* The binned update of sd_update (tuning mode 5) without any device
 * allocation, for callers that cannot allocate: an ingest thread on a
 * latency budget (cudaMalloc can synchronise the device and take
 * milliseconds) or a program whose device memory is owned entirely by
 * another allocator.  There is no counterpart in the paper; it is the same
 * Algorithm 1 as sd_update.
 *
 * Sets, for both directions of *p, the DHLA bits of n (src, dst) pairs.
 * `grid` is a caller-owned device DHLA of dirs * sd_grid_words(p) words in
 * the sd_get_grid layout (direction 0 first), 16-byte aligned; `pairs` holds
 * 2n device words, 4-byte aligned.  Runs on `cuda_stream` (NULL: the legacy
 * default stream) of the current device and returns once the work is queued.
 *
 * Scratch: a 16 MiB array inside the library (every GPU that loads the
 * library holds it until the process exits).  The first call on a device
 * looks up that array's address on the device, so make it before any stream
 * capture.  All calls share the array: calls whose work overlaps on the GPU
 * race and must be serialised by the caller.  Returns SD_ERR_TOO_LARGE when
 * the DHLA has more than 512 MiB (4096 slices of 128 KiB) or its bins would
 * not fit the scratch; SD_ERR_ARG for invalid parameters, or for a `grid` or
 * `pairs` that is not device (or managed) memory of the current device;
 * SD_ERR_CUDA when a CUDA call fails, or, with nothing queued, when the
 * calling thread already has a CUDA error pending from earlier work (that
 * error is left in place for the caller). */
int sd_update_noalloc(const sd_params *p, uint32_t *grid, const uint32_t *pairs, uint64_t n,
                      void *cuda_stream);

#ifdef __cplusplus
}
#endif

#endif /* SD_H */
