// sd_api.cu -- the C ABI declared in include/sd.h: handle lifetime, host
// ingest, and the orchestration of the close path.
//
// The host evaluates the few per-window scalars in double: Zmin and the
// integer hot threshold zhot (Algorithm 2), psi (Lemma 1 with the w(i)'
// average of §3.3), the largest SZ that Eq. 4 still reports (szmax), and
// Eq. 4 itself for each reported host.  These are evaluated exactly as the
// paper writes them, in IEEE double with step-by-step rounding
// (-ffp-contract=off), so every implementation that follows the same
// formulas with the same libm agrees bit for bit.  All per-pair, per-
// estimator and per-candidate work runs in the kernels.
#include <algorithm>
#include <atomic>
#include <chrono>
#include <cmath>
#include <cstdlib>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <memory>
#include <mutex>
#include <string>
#include <vector>

#include <nvtx3/nvToolsExt.h>

#include "sd.h"
#include "sd_common.cuh"

using namespace sd;

namespace {

thread_local std::string g_create_error;
std::atomic<uint64_t> g_launches{0};  // kernels launched by this library, all handles

void launched(uint64_t k) { g_launches.fetch_add(k, std::memory_order_relaxed); }

// An NVTX range over one entry point, so that profilers can attribute and
// filter the kernels of an update, a close or a merge (a no-op when no tool
// is attached).
struct NvtxRange {
    explicit NvtxRange(const char *name) { nvtxRangePushA(name); }
    ~NvtxRange() { nvtxRangePop(); }
    NvtxRange(const NvtxRange &) = delete;
    NvtxRange &operator=(const NvtxRange &) = delete;
};

// splitmix64 (Steele, Lea, Flood 2014): the published generator.
uint64_t splitmix64(uint64_t *state) {
    uint64_t z = (*state += 0x9E3779B97F4A7C15ull);
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

uint32_t inverse_odd(uint32_t a) {  // Newton: x <- x(2 - a x) doubles correct bits
    uint32_t x = a;
    for (int i = 0; i < 5; i++) x *= 2u - a * x;
    return x;
}

uint32_t ilog2(uint32_t v) {
    uint32_t l = 0;
    while ((1u << l) < v) l++;
    return l;
}

uint64_t next_pow2(uint64_t v) {
    uint64_t p = 1;
    while (p < v) p <<= 1;
    return p;
}

// Algorithm 2: Zmin = g e^(-theta/g); the largest integer z with z < Zmin.
int zhot_of(uint32_t g, double theta) {
    const double Zmin = (double)g * exp(-theta / (double)g);
    double f = floor(Zmin);
    if (f >= Zmin) f -= 1.0;
    if (f > (double)g) f = (double)g;
    if (f < -1.0) f = -1.0;
    return (int)f;
}

// Lemma 1 with w' the mean of w(i)' = -g 2^k ln(ZR(i)/(g 2^k)) (§3.3).
// -1 when a row is saturated.
double psi_of(uint32_t g, uint32_t r, uint32_t k, const unsigned long long *zr) {
    const double G = (double)g * (double)((uint64_t)1 << k);
    double wsum = 0.0;
    for (uint32_t i = 0; i < r; i++) {
        if (zr[i] == 0) return -1.0;
        const double wi = -G * log((double)zr[i] / G);
        wsum += wi;
    }
    const double w = wsum / (double)r;
    return 1.0 - exp(-w / G);
}

// Eq. 4: C(a0) = -g ln(SZ(a0) / (g - g psi^r)).
double eq4(uint32_t g, uint32_t r, double psi, uint32_t sz) {
    const double gd = (double)g;
    return -gd * log((double)sz / (gd - gd * pow(psi, (double)r)));
}

// Largest SZ in [0, g] that Algorithm 2 reports (C(SZ) >= theta); -1 if none.
// C decreases in SZ, so the reported values form a prefix [0, szmax].
int szmax_of(uint32_t g, uint32_t r, double psi, double theta) {
    auto pass = [&](uint32_t s) { return eq4(g, r, psi, s) >= theta; };
    if (!pass(0)) return -1;
    if (pass(g)) return (int)g;
    uint32_t lo = 0, hi = g;  // pass(lo), !pass(hi)
    while (hi - lo > 1) {
        const uint32_t mid = lo + (hi - lo) / 2;
        if (pass(mid)) lo = mid;
        else hi = mid;
    }
    return (int)lo;
}

struct LaunchKey {
    const void *fn;
    int dev, threads;
    size_t smem;
    int per_sm;
};
std::mutex g_launch_mu;
std::vector<LaunchKey> g_launch_cache;
std::vector<std::pair<std::pair<const void *, int>, size_t>> g_smem_set;  // (fn, dev) -> opted-in bytes

struct DeviceGuard {
    int prev = -1;
    explicit DeviceGuard(int dev) {
        if (cudaGetDevice(&prev) != cudaSuccess) prev = -1;
        if (prev != dev) cudaSetDevice(dev);
    }
    ~DeviceGuard() {
        int cur = -1;
        if (prev >= 0 && cudaGetDevice(&cur) == cudaSuccess && cur != prev) cudaSetDevice(prev);
    }
};

}  // namespace

// Per-window state carried between the close phases.
struct CloseState {
    uint32_t flags;
    RestoreArgs A;
    double psi[2];
    uint64_t nh[2];                        // hits per direction
    const unsigned long long *keys[2];     // their sorted keys in pinned host memory
};

// The report's hits: a plain growable array that is not zero-filled when it
// grows (every slot is written by the close before it is read).
class HitBuf {
  public:
    void clear() { n_ = 0; }
    size_t size() const { return n_; }
    bool empty() const { return n_ == 0; }
    sd_hit *data() { return buf_.get(); }
    sd_hit &operator[](size_t i) { return buf_[i]; }
    void truncate(size_t n) { n_ = n < n_ ? n : n_; }
    void grow_to(size_t n) {
        if (n > cap_) {
            size_t c = cap_ ? cap_ : 1024;
            while (c < n) c *= 2;
            std::unique_ptr<sd_hit[]> b(new sd_hit[c]);
            if (n_) std::memcpy(b.get(), buf_.get(), n_ * sizeof(sd_hit));
            buf_ = std::move(b);
            cap_ = c;
        }
        n_ = n;
    }

  private:
    std::unique_ptr<sd_hit[]> buf_;
    size_t n_ = 0, cap_ = 0;
};

constexpr uint32_t kBatchLanes = 4;  // concurrent member lanes of a plane-mode sd_update_many

struct sd_handle {
    sd_params p{};
    Geometry G{};
    Tuning T{};
    int num_sms = 0;
    int pageable_access = 0;  // kernels may read pageable host memory in place
    int zhot = -1;
    cudaStream_t stream = nullptr;
    bool own_stream = false;
    cudaStream_t copy_stream = nullptr;

    uint32_t *grid = nullptr;          // [dirs][r][2^k][g/32]
    StatBlock *st_d = nullptr;
    StatBlock *st_h = nullptr;         // pinned
    uint32_t *hotmap = nullptr;        // [dirs][r][2^k/32]
    uint32_t *he = nullptr;            // [dirs][2][2^k]
    uint32_t *cand = nullptr;          // [dirs][cand_cap]
    unsigned long long *hits = nullptr;   // [dirs][hits_cap]
    unsigned long long *hits_tmp = nullptr;  // [dirs][hits_cap]: scratch of the large-list sort
    unsigned long long *hits_h = nullptr; // pinned [dirs][kSortSmall]
    uint64_t cand_cap = 0, hits_cap = 0, report_cap = 0, pair_cap = 0;
    unsigned long long *big_h = nullptr;  // pinned [2][hits_cap]: large sorted hit lists
    void *ss_d = nullptr;                 // [2] sample-sort scratch (kSampleScratchBytes each)
    uint32_t *ss_flag_h = nullptr;        // pinned [2]: a sample sort fell short
    bool ss_check[2] = {false, false};    // ss_flag_h[d] is to be checked after the close's last sync
    HitBuf report;
    std::vector<double> est_tbl;
    uint64_t last_ncand[2] = {0, 0};
    bool have_close = false;
    CloseState cs{};

    // batched close (sd_close_many) driven by this handle: the jobs, and
    // every job's StatBlock and first hit keys gathered for one copy back
    CloseJob *cj_d = nullptr, *cj_h = nullptr;  // cj_h pinned
    StatBlock *cb_st_d = nullptr, *cb_st_h = nullptr;
    unsigned long long *cb_hits_d = nullptr, *cb_hits_h = nullptr;
    unsigned long long *cb_base_d = nullptr, *cb_base_h = nullptr;  // tile and candidate offsets
    FoldJob *fj_d = nullptr, *fj_h = nullptr;  // members' plane folds (fj_h pinned)
    uint32_t cj_cap = 0;

    // staged join (tuning restore = 1): all hot lists and the two
    // intermediate buffers, allocated on first use
    uint32_t *he_all = nullptr;
    unsigned long long *jsub = nullptr;  // [2][dirs][join_cap]
    uint64_t join_cap = 0;

    // binned update (mode 5): scratch sized for the current tuning
    uint32_t *bin_mem = nullptr;       // bins [S][cap], then count [S], then work [1]
    uint64_t bin_mem_words = 0;
    BinArgs bin{};

    // plane-binned update (mode 6): the plane-major DHLA copy (the handle's
    // DHLA is grid | planes^T; folded into grid before anything reads it)
    // and the per-plane counters, allocated on first use; the bins of its
    // own rounds (a batch it drives runs every member's rounds through
    // them), grown on demand
    uint32_t *planes = nullptr;
    uint32_t *plane_ctr = nullptr;     // cnt, prev, binoff, cap, unit_start, ctl
    uint32_t *plane_bins = nullptr;
    uint64_t plane_bins_words = 0;
    // a plane batch it drives: side streams, their bins and events (lane 0
    // is the handle's own stream and bins)
    cudaStream_t lane_stream[kBatchLanes - 1] = {};
    uint32_t *lane_bins[kBatchLanes - 1] = {};
    uint64_t lane_bins_words[kBatchLanes - 1] = {};
    cudaEvent_t lane_ev[kBatchLanes] = {};
    PlaneArgs pa{};                    // counters and plane copy (bins, tile, unit set per round)
    bool planes_dirty = false;
    bool grid_clean = false;           // the DHLA is all zero (reset, then plane updates only)
    uint64_t plane_prev_pairs = 0;     // pairs of the round whose counts are in prev (0: none)
    int plane_layout_view = -2;        // its directions (-1 both, else one)

    // key partition (sd_partition_pairs): per-part counts and cursors
    unsigned long long *part_d = nullptr;  // [2][1024]
    unsigned long long *part_h = nullptr;  // pinned [1024]

    // batched update (sd_update_many): link tables in two halves used by
    // alternate calls (a half is rewritten once the call two back has read
    // it, so consecutive calls do not wait for each other), an event per
    // half, and an event for stream joins
    LinkDesc *links_dev = nullptr;
    LinkDesc *links_h = nullptr;       // pinned
    uint32_t links_cap = 0;            // descriptors per half
    int links_half = 0;
    cudaEvent_t ev_links[2] = {nullptr, nullptr};
    cudaEvent_t ev_batch = nullptr;

    uint64_t stage_pairs = 0;
    uint32_t *dstage[2] = {nullptr, nullptr};
    uint32_t *hstage[2] = {nullptr, nullptr};  // pinned
    cudaEvent_t ev_h2d[2] = {nullptr, nullptr};
    cudaEvent_t ev_kern[2] = {nullptr, nullptr};
    uint64_t n_pairs = 0;
    std::string err;

    int fail(int code, const char *fmt, ...) {
        char buf[512];
        va_list ap;
        va_start(ap, fmt);
        vsnprintf(buf, sizeof buf, fmt, ap);
        va_end(ap);
        err = buf;
        return code;
    }
};

#define SD_CK(h, call)                                                                         \
    do {                                                                                       \
        cudaError_t e_ = (call);                                                               \
        if (e_ != cudaSuccess)                                                                 \
            return (h)->fail(e_ == cudaErrorMemoryAllocation ? SD_ERR_NOMEM : SD_ERR_CUDA,     \
                             "%s: %s (%s:%d)", #call, cudaGetErrorString(e_), __FILE__, __LINE__); \
    } while (0)

namespace sd {

cudaError_t prepare_launch(const void *kernel, int threads, size_t smem, int *per_sm) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    std::lock_guard<std::mutex> lock(g_launch_mu);
    for (const LaunchKey &k : g_launch_cache)
        if (k.fn == kernel && k.dev == dev && k.threads == threads && k.smem == smem) {
            *per_sm = k.per_sm;
            return cudaSuccess;
        }
    // dynamic shared memory beyond the default 48 KiB (counting the kernel's
    // static shared memory, which shares that limit) needs an opt-in
    cudaFuncAttributes fa;
    e = cudaFuncGetAttributes(&fa, kernel);
    if (e != cudaSuccess) return e;
    if (smem + fa.sharedSizeBytes > 48 * 1024) {
        size_t *have = nullptr;
        for (auto &p : g_smem_set)
            if (p.first.first == kernel && p.first.second == dev) have = &p.second;
        if (!have || *have < smem) {
            e = cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
            if (e != cudaSuccess) return e;
            if (have) *have = smem;
            else g_smem_set.push_back({{kernel, dev}, smem});
        }
    }
    int n = 0;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, kernel, threads, smem);
    if (e != cudaSuccess) return e;
    *per_sm = n > 0 ? n : 1;
    g_launch_cache.push_back({kernel, dev, threads, smem, *per_sm});
    return cudaSuccess;
}

}  // namespace sd

// Layout and hash constants of a DHLA with parameters *p (§3.1-3.2): per
// direction, A0, A1, B1 are the first three splitmix64 outputs for the state
// seed ^ (0x9E3779B97F4A7C15 (dir + 1)), with A0 and A1 made odd.
void sd::geometry_of(const sd_params *p, Geometry *out) {
    Geometry G;
    std::memset(&G, 0, sizeof G);
    G.g = p->g;
    G.r = p->r;
    G.k = p->k;
    G.alpha = p->alpha;
    G.dirs = p->dirs;
    G.lg = ilog2(p->g);
    G.wpc = p->g / 32;
    G.row_words = ((uint64_t)1 << p->k) * G.wpc;
    G.dir_words = (uint64_t)p->r * G.row_words;
    for (uint32_t d = 0; d < 2; d++) {
        uint64_t st = p->seed ^ (0x9E3779B97F4A7C15ull * (uint64_t)(d + 1));
        G.h[d].A0 = (uint32_t)splitmix64(&st) | 1u;
        G.h[d].A1 = splitmix64(&st) | 1ull;
        G.h[d].B1 = splitmix64(&st);
        G.h[d].A0inv = inverse_odd(G.h[d].A0);
    }
    *out = G;
}

extern "C" {

int sd_default_params(sd_params *p) {
    if (!p) return SD_ERR_ARG;
    std::memset(p, 0, sizeof *p);
    p->g = 512;
    p->r = 4;
    p->k = 16;
    p->alpha = 8;
    p->theta = 1024.0;
    p->seed = 0x5D5A0002ull;
    p->dirs = 2;
    p->device = 0;
    return SD_OK;
}

int sd_check_params(const sd_params *p) {
    if (!p) return SD_ERR_ARG;
    if (p->g < 32 || p->g > 4096 || (p->g & (p->g - 1))) return SD_ERR_ARG;
    if (p->r < 3 || p->r > (uint32_t)kMaxRows) return SD_ERR_ARG;
    if (p->k < 1 || p->k > 24) return SD_ERR_ARG;
    if (p->alpha < 1 || p->alpha > p->k) return SD_ERR_ARG;       // alpha <= k
    if ((p->r - 2) * p->alpha + p->k < 32) return SD_ERR_ARG;      // (r-2) alpha + k >= 32
    if (p->dirs < 1 || p->dirs > 2) return SD_ERR_ARG;
    if (!(p->theta > 0.0) || !std::isfinite(p->theta)) return SD_ERR_ARG;
    if (p->device < 0) return SD_ERR_ARG;
    return SD_OK;
}

uint64_t sd_grid_words(const sd_params *p) {
    if (sd_check_params(p) != SD_OK) return 0;
    return (uint64_t)p->r * ((uint64_t)1 << p->k) * (p->g / 32);
}

static void resolve_caps(const sd_params *p, uint64_t *pair_cap, uint64_t *cand_cap, uint64_t *hits_cap,
                         uint64_t *report_cap, uint64_t *stage) {
    *pair_cap = p->pair_cap ? p->pair_cap : (1ull << 32);
    *cand_cap = p->cand_cap ? p->cand_cap : (1ull << 20);
    *hits_cap = next_pow2(*cand_cap);
    *report_cap = p->report_cap ? p->report_cap : (uint64_t)p->dirs * *cand_cap;
    // host-ingest chunks: 2^22 pairs keep the last chunk's kernels short; a
    // DHLA larger than L2 takes 2^24 (each chunk is one binning round, and
    // every round reads and writes such a DHLA in DRAM once)
    const uint64_t dhla_bytes = (uint64_t)p->dirs * p->r * ((uint64_t)1 << p->k) * (p->g / 8);
    *stage = p->stage_pairs ? p->stage_pairs : (dhla_bytes > (64ull << 20) ? (1ull << 24) : (1ull << 22));
}

}  // extern "C"

// Words of one bit plane (r estimators' bit b), 16-byte aligned.
static uint32_t plane_words(const Geometry &G) {
    return (uint32_t)((((uint64_t)G.r << G.k) / 32 + 3) & ~3ull);
}

// Most shared memory one bit plane may take in k_plane_apply.
constexpr uint64_t kPlaneSmemMax = 192 * 1024;

static bool plane_fits(const Geometry &G) { return (uint64_t)plane_words(G) * 4 <= kPlaneSmemMax; }

// Bins of a plane round of `round` pairs over G's directions: each plane's
// bin holds a count (the previous round's, possibly scaled; exact for a
// counted round) plus an eighth and 32 slots, rounded up to 4, and scaling
// adds at most one slot per plane; so the total stays below keys + keys/8 +
// 40 per plane.
static uint64_t plane_bin_words(const Geometry &G, uint64_t round) {
    const uint64_t keys = (uint64_t)G.dirs * round;
    return keys + keys / 8 + 40ull * G.dirs * G.g;
}
// Words of a handle's plane state: the plane-major copy and the counters
// (cnt, prev, cap: nbins each; binoff, unit_start: nbins + 1; ctl: 4).
constexpr uint64_t kPlaneCtlWords = 4;
static uint64_t plane_ctr_words(uint32_t nbins) { return 5ull * nbins + 2 + kPlaneCtlWords; }
static uint64_t plane_state_words(const Geometry &G) {
    const uint64_t nb = (uint64_t)G.dirs * G.g;
    return nb * plane_words(G) + plane_ctr_words((uint32_t)nb);
}

extern "C" {

uint64_t sd_device_bytes(const sd_params *p) {
    if (sd_check_params(p) != SD_OK) return 0;
    uint64_t pc, cc, hc, rc, sp;
    resolve_caps(p, &pc, &cc, &hc, &rc, &sp);
    const uint64_t cells = (uint64_t)p->r << p->k;
    (void)sp;  // the host-pointer staging is allocated on first use, not counted
    Geometry G;
    geometry_of(p, &G);
    const uint64_t planes = plane_fits(G) ? plane_state_words(G) * 4 : 0;  // default mode 6
    return (uint64_t)p->dirs * (sd_grid_words(p) * 4 + cells / 8 + 2 * ((uint64_t)4 << p->k) + cc * 4 + 2 * hc * 8) +
           sizeof(StatBlock) + planes;
}

static void release(sd_handle *h) {
    if (h->stream) cudaStreamSynchronize(h->stream);
    if (h->copy_stream) cudaStreamSynchronize(h->copy_stream);
    cudaFree(h->grid);
    cudaFree(h->st_d);
    cudaFree(h->hotmap);
    cudaFree(h->he);
    cudaFree(h->cand);
    cudaFree(h->hits);
    cudaFree(h->hits_tmp);
    cudaFree(h->bin_mem);
    cudaFree(h->planes);
    cudaFree(h->plane_ctr);
    cudaFree(h->plane_bins);
    for (uint32_t l = 0; l + 1 < kBatchLanes; l++) {
        if (h->lane_stream[l]) cudaStreamSynchronize(h->lane_stream[l]);
        cudaFree(h->lane_bins[l]);
        if (h->lane_stream[l]) cudaStreamDestroy(h->lane_stream[l]);
    }
    for (uint32_t l = 0; l < kBatchLanes; l++)
        if (h->lane_ev[l]) cudaEventDestroy(h->lane_ev[l]);
    cudaFree(h->part_d);
    cudaFreeHost(h->part_h);
    cudaFree(h->he_all);
    cudaFree(h->jsub);
    cudaFree(h->cj_d);
    cudaFreeHost(h->cj_h);
    cudaFree(h->cb_st_d);
    cudaFreeHost(h->cb_st_h);
    cudaFree(h->cb_hits_d);
    cudaFreeHost(h->cb_hits_h);
    cudaFree(h->cb_base_d);
    cudaFreeHost(h->cb_base_h);
    cudaFree(h->fj_d);
    cudaFreeHost(h->fj_h);
    cudaFreeHost(h->st_h);
    cudaFreeHost(h->hits_h);
    cudaFreeHost(h->big_h);
    cudaFree(h->ss_d);
    cudaFreeHost(h->ss_flag_h);
    for (int b = 0; b < 2; b++) {
        cudaFree(h->dstage[b]);
        cudaFreeHost(h->hstage[b]);
        if (h->ev_h2d[b]) cudaEventDestroy(h->ev_h2d[b]);
        if (h->ev_kern[b]) cudaEventDestroy(h->ev_kern[b]);
    }
    cudaFree(h->links_dev);
    cudaFreeHost(h->links_h);
    if (h->ev_batch) cudaEventDestroy(h->ev_batch);
    for (int b = 0; b < 2; b++)
        if (h->ev_links[b]) cudaEventDestroy(h->ev_links[b]);
    if (h->copy_stream) cudaStreamDestroy(h->copy_stream);
    if (h->own_stream && h->stream) cudaStreamDestroy(h->stream);
}

static int create_impl(const sd_params *p, sd_handle *h) {
    h->p = *p;
    geometry_of(p, &h->G);
    const Geometry &G = h->G;
    // binned update, 128 KiB slices, 1024-pair tiles, 2^24-pair rounds (autotuned on GB300);
    // a DHLA of 1024 slices or more takes 2048-pair tiles, so that each
    // slice's run in a tile stays long enough for coalesced bin writes
    // (autotuned on the 2 x 128 MiB stress sketch: 50 ms vs 72 ms per 2^30 pairs)
    h->T = Tuning{5, 512, 0, 2, 13, 15, 1024, 24, 100, 0, 8192, 8192, 26, 14};
    if ((uint64_t)p->dirs * G.dir_words >= (1ull << 25) && p->dirs * p->r <= 8) h->T.bin_tile_pairs = 2048;
    // binned by estimator bit wherever one bit plane fits a block's shared
    // memory (r 2^k bits: every workload of the scope table), with tiles of
    // 8192 pairs and rounds of 2^26 (measured on GB300 over tiles 1024-8192,
    // rounds 2^22-2^26 and apply units 2^13-2^16: 0.67 ms per 2^26-pair core
    // window, against 0.79 ms at 4096 / 2^24 and 1.2 ms at 2048 / 2^24);
    // 4096-pair tiles where 8192 would not fit shared memory
    if (plane_fits(G)) h->T.mode = 6;
    // apply units of at least twice a plane's words in keys: every unit ORs
    // its whole plane into the plane copy, which for planes beyond 32 KiB
    // (k >= 18: a copy larger than L2) goes to DRAM
    h->T.plane_unit_log2 = std::max<uint32_t>(14u, ilog2(plane_words(G)) + 1u);
    if (plane_bin_smem_bytes(h->T.plane_tile_pairs, G.dirs, G.dirs * G.g) > 200 * 1024) h->T.plane_tile_pairs = 4096;
    h->zhot = zhot_of(p->g, p->theta);
    resolve_caps(p, &h->pair_cap, &h->cand_cap, &h->hits_cap, &h->report_cap, &h->stage_pairs);

    SD_CK(h, cudaSetDevice(p->device));
    SD_CK(h, cudaDeviceGetAttribute(&h->num_sms, cudaDevAttrMultiProcessorCount, p->device));
    SD_CK(h, cudaDeviceGetAttribute(&h->pageable_access, cudaDevAttrPageableMemoryAccess, p->device));
    if (p->cuda_stream) {
        h->stream = (cudaStream_t)p->cuda_stream;
    } else {
        SD_CK(h, cudaStreamCreateWithFlags(&h->stream, cudaStreamNonBlocking));
        h->own_stream = true;
    }
    // the side stream (staged host copies, and the close's kernels) has the
    // device's highest priority: a close is scheduled ahead of other queued
    // work, e.g. another window's update, whenever an SM frees up
    int prio_least = 0, prio_greatest = 0;
    SD_CK(h, cudaDeviceGetStreamPriorityRange(&prio_least, &prio_greatest));
    SD_CK(h, cudaStreamCreateWithPriority(&h->copy_stream, cudaStreamNonBlocking, prio_greatest));
    for (int b = 0; b < 2; b++) {
        SD_CK(h, cudaEventCreateWithFlags(&h->ev_h2d[b], cudaEventDisableTiming));
        SD_CK(h, cudaEventCreateWithFlags(&h->ev_kern[b], cudaEventDisableTiming));
    }
    SD_CK(h, cudaEventCreateWithFlags(&h->ev_batch, cudaEventDisableTiming));
    for (int b = 0; b < 2; b++) SD_CK(h, cudaEventCreateWithFlags(&h->ev_links[b], cudaEventDisableTiming));
    const uint64_t words = (uint64_t)p->dirs * G.dir_words;
    const uint64_t nw = ((uint64_t)1 << p->k) >> 5;
    SD_CK(h, cudaMalloc(&h->grid, words * 4));
    SD_CK(h, cudaMalloc(&h->st_d, sizeof(StatBlock)));
    SD_CK(h, cudaMalloc(&h->hotmap, (uint64_t)p->dirs * p->r * nw * 4));
    SD_CK(h, cudaMalloc(&h->he, (uint64_t)p->dirs * 2 * ((uint64_t)4 << p->k)));
    SD_CK(h, cudaMalloc(&h->cand, (uint64_t)p->dirs * h->cand_cap * 4));
    SD_CK(h, cudaMalloc(&h->hits, (uint64_t)p->dirs * h->hits_cap * 8));
    SD_CK(h, cudaMalloc(&h->hits_tmp, (uint64_t)p->dirs * h->hits_cap * 8));
    SD_CK(h, cudaMallocHost(&h->st_h, sizeof(StatBlock)));
    SD_CK(h, cudaMallocHost(&h->hits_h, (uint64_t)2 * kSortSmall * 8));
    SD_CK(h, launch_reset(h->grid, words, h->st_d, h->num_sms, h->stream));
    SD_CK(h, cudaStreamSynchronize(h->stream));
    h->grid_clean = true;
    return SD_OK;
}

int sd_create(const sd_params *p, sd_handle **out) {
    if (!out) return SD_ERR_ARG;
    if (sd_check_params(p) != SD_OK) {
        g_create_error = "sd_create: invalid parameters (see sd_check_params)";
        return SD_ERR_ARG;
    }
    sd_handle *h = new (std::nothrow) sd_handle();
    if (!h) {
        g_create_error = "sd_create: out of host memory";
        return SD_ERR_NOMEM;
    }
    int prev = -1;
    cudaGetDevice(&prev);
    const int rc = create_impl(p, h);
    if (prev >= 0) cudaSetDevice(prev);
    if (rc != SD_OK) {
        g_create_error = h->err;
        release(h);
        delete h;
        return rc;
    }
    *out = h;
    return SD_OK;
}

static int ensure_staging(sd_handle *h) {
    if (h->dstage[0]) return SD_OK;
    for (int b = 0; b < 2; b++) {
        SD_CK(h, cudaMalloc(&h->dstage[b], h->stage_pairs * 8));
        SD_CK(h, cudaMallocHost(&h->hstage[b], h->stage_pairs * 8));
    }
    return SD_OK;
}

// Geometry of the binned update for the current tuning: slices of
// 2^slice_log2 words (at most 4096 of them, so a (slice, rank) pair packs in
// 32 bits), bins sized for 2^chunk_log2 pairs per round plus the slack.
// Returns false when the DHLA is too large for binning.
static bool bin_layout(const sd_handle *h, BinArgs *B, uint64_t *words) {
    const Geometry &G = h->G;
    const uint64_t total = (uint64_t)G.dirs * G.dir_words;
    uint32_t sl = h->T.bin_slice_log2;
    while (((total + (1ull << sl) - 1) >> sl) > 4096 && sl < 15) sl++;
    const uint64_t S = (total + (1ull << sl) - 1) >> sl;
    if (S > 4096 || (1ull << sl) > total) return false;
    const uint64_t chunk = 1ull << h->T.bin_chunk_log2;
    const uint64_t mean = (chunk * G.dirs * G.r + S - 1) / S;
    uint64_t cap = mean + mean * h->T.bin_slack_pct / 100 + 256;
    cap = (cap + 3) & ~3ull;
    if (cap > 0xFFFFFFFFull) return false;
    std::memset(B, 0, sizeof *B);
    B->S = (uint32_t)S;
    B->slice_log2 = sl;
    B->cap = (uint32_t)cap;
    B->tile_pairs = h->T.bin_tile_pairs;
    B->total_words = total;
    *words = S * cap + S + 4;
    return true;
}

// Bin scratch for S slices of `cap` entries (grows, never shrinks).
static int ensure_bin_mem(sd_handle *h, BinArgs &B) {
    const uint64_t words = (uint64_t)B.S * B.cap + B.S + 4;
    if (words > h->bin_mem_words) {
        SD_CK(h, cudaStreamSynchronize(h->stream));
        cudaFree(h->bin_mem);
        h->bin_mem = nullptr;
        h->bin_mem_words = 0;
        SD_CK(h, cudaMalloc(&h->bin_mem, words * 4));
        h->bin_mem_words = words;
        SD_CK(h, cudaMemsetAsync(h->bin_mem + (uint64_t)B.S * B.cap, 0, ((uint64_t)B.S + 4) * 4, h->stream));
    } else if (B.S != h->bin.S || B.cap != h->bin.cap) {
        SD_CK(h, cudaMemsetAsync(h->bin_mem + (uint64_t)B.S * B.cap, 0, ((uint64_t)B.S + 4) * 4, h->stream));
    }
    B.bins = h->bin_mem;
    B.count = h->bin_mem + (uint64_t)B.S * B.cap;
    B.work = B.count + B.S;
    h->bin = B;
    return SD_OK;
}

static int ensure_bins(sd_handle *h, bool *ok) {
    BinArgs B;
    uint64_t words = 0;
    *ok = bin_layout(h, &B, &words);
    if (!*ok) return SD_OK;
    return ensure_bin_mem(h, B);
}

// A scaled layout needs a previous round of at least this many pairs per
// plane of a direction (64 keys per plane on average), else the round is
// counted exactly.
constexpr uint64_t kPlaneScaleMinPerPlane = 64;

// The plane copy (zero) and the counters (zero: no layout yet), once.
static int ensure_plane_state(sd_handle *h) {
    if (!h->planes) {
        const uint32_t nb = h->G.dirs * h->G.g;
        const uint64_t pw = (uint64_t)nb * plane_words(h->G), cw = plane_ctr_words(nb);
        SD_CK(h, cudaMalloc(&h->planes, pw * 4));
        SD_CK(h, cudaMalloc(&h->plane_ctr, cw * 4));
        SD_CK(h, cudaMemsetAsync(h->planes, 0, pw * 4, h->stream));
        SD_CK(h, cudaMemsetAsync(h->plane_ctr, 0, cw * 4, h->stream));
        PlaneArgs &P = h->pa;
        std::memset(&P, 0, sizeof P);
        P.nbins = nb;
        P.ps = plane_words(h->G);
        P.planes = h->planes;
        uint32_t *c = h->plane_ctr;
        P.cnt = c;
        P.prev = c + nb;
        P.cap = c + 2 * nb;
        P.binoff = c + 3 * nb;
        P.unit_start = c + 4 * nb + 1;
        P.ctl = c + 5 * nb + 2;
        h->plane_prev_pairs = 0;
        h->plane_layout_view = -2;
    }
    return SD_OK;
}

// owner's bins, at least `words` of them (grown once the rounds that read
// the old ones are done)
static int ensure_plane_bins(sd_handle *owner, uint64_t words) {
    if (words <= owner->plane_bins_words) return SD_OK;
    SD_CK(owner, cudaStreamSynchronize(owner->stream));
    cudaFree(owner->plane_bins);
    owner->plane_bins = nullptr;
    owner->plane_bins_words = 0;
    SD_CK(owner, cudaMalloc(&owner->plane_bins, words * 4));
    owner->plane_bins_words = words;
    return SD_OK;
}

// Algorithm 1 binned by plane over n device pairs of h, in rounds of at
// most `round` pairs through `bins` (bin_words of them, at least the bins
// of one round), on stream s; failures are reported on `rep`.  A round
// reuses the layout the previous round of the same directions left when it
// is no larger than that round and that layout fits the bins; a round of
// another size is laid out from the previous counts scaled to its size when
// that round had enough pairs; any other round is counted exactly.
static int plane_rounds(sd_handle *h, const uint32_t *pairs, uint64_t n, int dir, uint32_t *bins,
                        uint64_t bin_words, uint64_t round, cudaStream_t s, sd_handle *rep) {
    Geometry G = h->G;
    PlaneArgs P = h->pa;
    P.bins = bins;
    P.unit = 1u << h->T.plane_unit_log2;
    P.tile_pairs = h->T.plane_tile_pairs;
    if (dir >= 0) {  // one direction's hash constants, counters and planes
        G.dirs = 1;
        G.h[0] = h->G.h[dir];
        P.nbins = h->G.g;
        P.planes += (uint64_t)dir * h->G.g * P.ps;
    }
    if (plane_bin_words(G, std::min(round, n)) > bin_words)
        return rep->fail(SD_ERR_ARG, "plane update: %llu bin words for rounds of %llu pairs",
                         (unsigned long long)bin_words, (unsigned long long)round);
    for (uint64_t off = 0; off < n; off += round) {
        const uint64_t m = std::min(round, n - off);
        const uint64_t prev = h->plane_layout_view == dir ? h->plane_prev_pairs : 0;
        PlaneLayout L = kLayoutCount;
        if (prev && m <= prev && plane_bin_words(G, prev) <= bin_words) L = kLayoutReuse;
        else if (prev >= kPlaneScaleMinPerPlane * G.g) L = kLayoutScale;
        SD_CK(rep, launch_plane_round(pairs + 2 * off, m, G, P, h->num_sms, s, L, prev));
        launched(L == kLayoutReuse ? 2 : 3);
        h->plane_prev_pairs = m;
        h->plane_layout_view = dir;
    }
    h->planes_dirty = true;
    return SD_OK;
}

// grid |= planes^T and planes = 0 (stream-ordered), when updates of the
// plane-binned mode are pending.
static int fold_planes(sd_handle *h) {
    if (!h->planes_dirty) return SD_OK;
    const FoldJob job{h->grid, h->planes, h->grid_clean ? 1u : 0u, h->zhot, nullptr, nullptr};
    SD_CK(h, launch_plane_fold(job, nullptr, 1, h->G, h->pa.ps, h->num_sms, h->stream));
    launched(1);
    h->planes_dirty = false;
    h->grid_clean = false;
    return SD_OK;
}

// Algorithm 1 over n device-resident pairs, with the handle's tuning: both
// directions of (src, dst) pairs (dir < 0), or direction dir alone of
// (key, peer) pairs.  A single direction runs the same kernels on a
// one-direction view of the DHLA: that direction's hash constants and its
// part of the DHLA (and of the plane copy).
static int update_device(sd_handle *h, const uint32_t *pairs, uint64_t n, int dir = -1) {
    Geometry G = h->G;
    uint32_t *grid = h->grid;
    if (dir >= 0) {
        G.dirs = 1;
        G.h[0] = h->G.h[dir];
        grid += (uint64_t)dir * h->G.dir_words;
    }
    if (h->T.mode == 6) {
        int rc = ensure_plane_state(h);
        if (rc != SD_OK) return rc;
        const uint64_t round = 1ull << h->T.plane_round_log2;
        rc = ensure_plane_bins(h, plane_bin_words(h->G, round));
        if (rc != SD_OK) return rc;
        return plane_rounds(h, pairs, n, dir, h->plane_bins, h->plane_bins_words, round, h->stream, h);
    }
    h->grid_clean = false;  // the other modes set bits in the DHLA itself
    if (h->T.mode == 5) {
        bool ok = false;
        const int rc = ensure_bins(h, &ok);
        if (rc != SD_OK) return rc;
        if (ok) {
            BinArgs B = h->bin;
            if (dir >= 0) {  // the same bins and slice size over one direction's words
                B.total_words = h->G.dir_words;
                B.S = (uint32_t)((B.total_words + (1ull << B.slice_log2) - 1) >> B.slice_log2);
            }
            const uint64_t chunk = 1ull << h->T.bin_chunk_log2;
            for (uint64_t off = 0; off < n; off += chunk) {
                const uint64_t m = std::min(chunk, n - off);
                SD_CK(h, launch_binned_chunk(pairs + 2 * off, m, grid, G, B, h->num_sms, h->stream));
                launched(2);
            }
            return SD_OK;
        }
        Tuning T = h->T;  // DHLA too large to bin: test-then-set
        T.mode = 1;
        SD_CK(h, launch_update(pairs, n, grid, G, T, h->num_sms, h->stream));
        launched(1);
        return SD_OK;
    }
    SD_CK(h, launch_update(pairs, n, grid, G, h->T, h->num_sms, h->stream));
    launched(1);
    return SD_OK;
}

// sd_update and sd_update_dir: device pointers in place, pageable host
// memory in place where the device reads it, other host memory through the
// pinned double-buffered staging.
static int update_any(sd_handle *h, const uint32_t *pairs, uint64_t n, int dir, const char *who) {
    if (!pairs) return h->fail(SD_ERR_ARG, "%s: pairs is NULL", who);
    if ((uintptr_t)pairs & 3u) return h->fail(SD_ERR_ARG, "%s: pairs is not 4-byte aligned", who);
    DeviceGuard dg(h->p.device);
    cudaPointerAttributes attr;
    if (cudaPointerGetAttributes(&attr, pairs) != cudaSuccess) {
        cudaGetLastError();
        attr.type = cudaMemoryTypeUnregistered;
    }
    const uint64_t counted = dir <= 0 ? n : 0;  // a window's pairs: those of direction 0
    if (attr.type == cudaMemoryTypeDevice || attr.type == cudaMemoryTypeManaged) {
        if (attr.type == cudaMemoryTypeDevice && attr.device != h->p.device)
            return h->fail(SD_ERR_ARG, "%s: pairs live on device %d, handle on %d", who, attr.device, h->p.device);
        const int rc = update_device(h, pairs, n, dir);
        if (rc != SD_OK) return rc;
        h->n_pairs += counted;
        return SD_OK;
    }
    const bool pinned = attr.type == cudaMemoryTypeHost;
    if (!pinned && h->pageable_access) {
        // pageable memory the GPU reads in place (coherent link): no staging;
        // the caller may reuse the buffer once the kernels are done
        const int rc = update_device(h, pairs, n, dir);
        if (rc != SD_OK) return rc;
        SD_CK(h, cudaStreamSynchronize(h->stream));
        h->n_pairs += counted;
        return SD_OK;
    }
    // host memory: chunked, double-buffered H2D overlapped with the kernel
    const int rc = ensure_staging(h);
    if (rc != SD_OK) return rc;
    uint64_t c = 0;
    for (uint64_t off = 0; off < n; off += h->stage_pairs, c++) {
        const uint64_t m = std::min(h->stage_pairs, n - off);
        const int b = (int)(c & 1);
        const void *src = pairs + 2 * off;
        SD_CK(h, cudaStreamWaitEvent(h->copy_stream, h->ev_kern[b], 0));
        if (!pinned) {
            SD_CK(h, cudaEventSynchronize(h->ev_h2d[b]));
            std::memcpy(h->hstage[b], src, m * 8);
            src = h->hstage[b];
        }
        SD_CK(h, cudaMemcpyAsync(h->dstage[b], src, m * 8, cudaMemcpyHostToDevice, h->copy_stream));
        SD_CK(h, cudaEventRecord(h->ev_h2d[b], h->copy_stream));
        SD_CK(h, cudaStreamWaitEvent(h->stream, h->ev_h2d[b], 0));
        const int urc = update_device(h, h->dstage[b], m, dir);
        if (urc != SD_OK) return urc;
        SD_CK(h, cudaEventRecord(h->ev_kern[b], h->stream));
    }
    // the caller may reuse a pinned buffer only once its copies are done
    if (pinned) SD_CK(h, cudaEventSynchronize(h->ev_h2d[(c - 1) & 1]));
    h->n_pairs += counted;
    return SD_OK;
}

int sd_update(sd_handle *h, const uint32_t *pairs, uint64_t n) {
    NvtxRange nvtx("sd_update");
    if (!h) return SD_ERR_ARG;
    if (n == 0) return SD_OK;
    return update_any(h, pairs, n, -1, "sd_update");
}

int sd_update_dir(sd_handle *h, uint32_t dir, const uint32_t *pairs, uint64_t n) {
    NvtxRange nvtx("sd_update_dir");
    if (!h) return SD_ERR_ARG;
    if (dir >= h->G.dirs) return h->fail(SD_ERR_ARG, "sd_update_dir: direction %u of a %u-direction handle", dir,
                                          h->G.dirs);
    if (n == 0) return SD_OK;
    return update_any(h, pairs, n, (int)dir, "sd_update_dir");
}

// Layout of a batched update driven by h (sd_update_many): slices per
// member DHLA, slice size, bin capacity per slice for a given member share,
// and the members a round of full shares (one chunk each) holds.  A round is
// bounded by 4096 slices and by the tuning's bin_batch_mib of bins; each
// member's apply sweeps its whole DHLA once per round, so shares are as long
// as the bins allow.  False when h does not bin.
struct BatchLayout {
    uint32_t S_link, sl, per_group;  // per_group: members of a round of full chunks
    uint64_t cap_link;               // bin capacity per slice for a full chunk
    uint64_t bin_bytes;              // bins one round may use
    uint64_t upd, slack;
    // bin capacity per slice when the largest member share of a round is `take` pairs
    uint64_t cap_for(uint64_t take) const {
        const uint64_t mean = (take * upd + S_link - 1) / S_link;
        return ((mean + mean * slack / 100 + 256) + 3) & ~3ull;
    }
};
static bool batch_layout(const sd_handle *h, BatchLayout *L) {
    BinArgs B;
    uint64_t words = 0;
    // a batch bins by DHLA slice (one slice range per member); handles in
    // either binned mode take part
    if ((h->T.mode != 5 && h->T.mode != 6) || !bin_layout(h, &B, &words)) return false;
    L->S_link = B.S;
    L->sl = B.slice_log2;
    L->upd = (uint64_t)h->p.dirs * h->p.r;
    L->slack = h->T.bin_slack_pct;
    L->bin_bytes = (uint64_t)h->T.bin_batch_mib << 20;
    L->cap_link = L->cap_for(1ull << h->T.bin_chunk_log2);
    if (L->cap_link > 0xFFFFFFFFull) return false;  // BinArgs.cap is 32-bit
    const uint64_t by_mem = L->bin_bytes / std::max<uint64_t>(1, (uint64_t)L->S_link * L->cap_link * 4);
    L->per_group = (uint32_t)std::max<uint64_t>(1, std::min<uint64_t>(4096u / L->S_link, by_mem));
    return true;
}

// Lanes of a plane batch driven by d over `members` members: as many bin
// buffers of one round as bin_batch_mib holds, at most kBatchLanes and one
// per member.
static uint32_t plane_batch_lanes(const sd_handle *d, uint64_t members) {
    const uint64_t bytes = plane_bin_words(d->G, 1ull << d->T.plane_round_log2) * 4;
    const uint64_t budget = (uint64_t)d->T.bin_batch_mib << 20;
    uint64_t lanes = budget / std::max<uint64_t>(1, bytes);
    lanes = std::min<uint64_t>(std::min<uint64_t>(lanes, kBatchLanes), members);
    return (uint32_t)std::max<uint64_t>(1, lanes);
}

uint64_t sd_scratch_bytes(const sd_handle *h, uint32_t links) {
    if (!h) return 0;
    BinArgs B;
    uint64_t words = 0;
    // plane mode: the bins of one round, for the handle's own rounds and for
    // every member's rounds of a batch it drives
    if (h->T.mode == 6)
        return plane_bin_words(h->G, 1ull << h->T.plane_round_log2) * 4 * (links <= 1 ? 1 : plane_batch_lanes(h, links));
    if ((h->T.mode != 5 && h->T.mode != 6) || !bin_layout(h, &B, &words)) return 0;
    if (links <= 1) return words * 4;
    BatchLayout L;
    if (!batch_layout(h, &L)) return words * 4;
    // a round holds as many members as its bins allow at their actual
    // shares, so the bins reach the byte bound whenever that bound binds
    const uint64_t m = std::min<uint64_t>(links, 4096u / L.S_link);
    const uint64_t S = m * L.S_link;
    const uint64_t full = S * L.cap_link * 4;
    return std::max<uint64_t>(words * 4, std::min<uint64_t>(full, std::max<uint64_t>(L.bin_bytes, (uint64_t)L.S_link * L.cap_link * 4)) + (S + 4) * 4);
}

// Whether member h (pairs p) joins a batch driven by d: device-resident
// pairs on d's device, d's DHLA shape, and not already in the batch.
static bool batch_member(const sd_handle *d, const sd_handle *h, const uint32_t *p, uint64_t n,
                         sd_handle *const *hs, const std::vector<uint32_t> &batch) {
    const sd_params &P = d->p;
    bool ok = n > 0 && p && !((uintptr_t)p & 3u) && h->p.g == P.g && h->p.r == P.r && h->p.k == P.k &&
              h->p.alpha == P.alpha && h->p.dirs == P.dirs && h->p.device == P.device;
    for (uint32_t q : batch)
        if (hs[q] == h) ok = false;
    if (ok) {
        cudaPointerAttributes attr;
        if (cudaPointerGetAttributes(&attr, p) != cudaSuccess) {
            cudaGetLastError();
            ok = false;
        } else {
            ok = attr.type == cudaMemoryTypeDevice && attr.device == P.device;
        }
    }
    return ok;
}

// Side lanes 1 .. lanes - 1 of d: a stream, an event and `words` of bins each.
static int ensure_lanes(sd_handle *d, uint32_t lanes, uint64_t words) {
    if (!d->lane_ev[0]) SD_CK(d, cudaEventCreateWithFlags(&d->lane_ev[0], cudaEventDisableTiming));
    for (uint32_t l = 1; l < lanes; l++) {
        if (!d->lane_stream[l - 1]) {
            SD_CK(d, cudaStreamCreateWithFlags(&d->lane_stream[l - 1], cudaStreamNonBlocking));
            SD_CK(d, cudaEventCreateWithFlags(&d->lane_ev[l], cudaEventDisableTiming));
        }
        if (d->lane_bins_words[l - 1] < words) {
            SD_CK(d, cudaStreamSynchronize(d->lane_stream[l - 1]));
            cudaFree(d->lane_bins[l - 1]);
            d->lane_bins[l - 1] = nullptr;
            d->lane_bins_words[l - 1] = 0;
            SD_CK(d, cudaMalloc(&d->lane_bins[l - 1], words * 4));
            d->lane_bins_words[l - 1] = words;
        }
    }
    return SD_OK;
}

// sd_update_many with d in mode 6: each member in mode 6 runs its plane
// rounds through one lane's bins on that lane's stream; the members are
// dealt to the lanes largest first, each to the lane with the fewest pairs
// so far, and each lane takes its members one after another.
static int update_many_planes(sd_handle *const *hs, const uint32_t *const *pairs, const uint64_t *ns,
                              uint32_t count) {
    sd_handle *d = hs[0];
    std::vector<uint32_t> batch;
    for (uint32_t i = 0; i < count; i++) {
        if (hs[i]->T.mode == 6 && batch_member(d, hs[i], pairs[i], ns[i], hs, batch)) {
            batch.push_back(i);
        } else {
            const int rc = sd_update(hs[i], pairs[i], ns[i]);
            if (rc != SD_OK) return rc;
        }
    }
    if (batch.empty()) return SD_OK;
    const uint64_t round = 1ull << d->T.plane_round_log2;
    const uint64_t words = plane_bin_words(d->G, round);
    const uint32_t lanes = plane_batch_lanes(d, batch.size());
    int rc = ensure_plane_bins(d, words);
    if (rc == SD_OK) rc = ensure_lanes(d, lanes, words);
    if (rc != SD_OK) return rc;
    // each member's state (zeroed on its own stream when new) and earlier
    // work come first
    for (uint32_t q : batch) {
        sd_handle *h = hs[q];
        if ((rc = ensure_plane_state(h)) != SD_OK) return rc;
        if (h == d || h->stream == d->stream) continue;
        SD_CK(h, cudaEventRecord(h->ev_batch, h->stream));
        SD_CK(d, cudaStreamWaitEvent(d->stream, h->ev_batch, 0));
    }
    std::vector<uint32_t> order(batch);
    std::stable_sort(order.begin(), order.end(), [&](uint32_t x, uint32_t y) { return ns[x] > ns[y]; });
    std::vector<uint64_t> load(lanes, 0);
    std::vector<uint32_t> lane_of(count, 0);
    for (uint32_t q : order) {
        const uint32_t l = (uint32_t)(std::min_element(load.begin(), load.end()) - load.begin());
        lane_of[q] = l;
        load[l] += ns[q];
    }
    if (lanes > 1) {
        SD_CK(d, cudaEventRecord(d->lane_ev[0], d->stream));
        for (uint32_t l = 1; l < lanes; l++) SD_CK(d, cudaStreamWaitEvent(d->lane_stream[l - 1], d->lane_ev[0], 0));
    }
    for (uint32_t q : order) {
        const uint32_t l = lane_of[q];
        cudaStream_t st = l ? d->lane_stream[l - 1] : d->stream;
        uint32_t *bins = l ? d->lane_bins[l - 1] : d->plane_bins;
        const uint64_t bw = l ? d->lane_bins_words[l - 1] : d->plane_bins_words;
        rc = plane_rounds(hs[q], pairs[q], ns[q], -1, bins, bw, round, st, d);
        if (rc != SD_OK) return rc;
    }
    for (uint32_t l = 1; l < lanes; l++) {
        SD_CK(d, cudaEventRecord(d->lane_ev[l], d->lane_stream[l - 1]));
        SD_CK(d, cudaStreamWaitEvent(d->stream, d->lane_ev[l], 0));
    }
    // later work on each member waits for the batch
    SD_CK(d, cudaEventRecord(d->ev_batch, d->stream));
    for (uint32_t q : batch) {
        sd_handle *h = hs[q];
        h->n_pairs += ns[q];
        if (h == d || h->stream == d->stream) continue;
        SD_CK(h, cudaStreamWaitEvent(h->stream, d->ev_batch, 0));
    }
    return SD_OK;
}

int sd_update_many(sd_handle *const *hs, const uint32_t *const *pairs, const uint64_t *ns, uint32_t count) {
    NvtxRange nvtx("sd_update_many");
    if (!count) return SD_OK;
    if (!hs || !pairs || !ns) return SD_ERR_ARG;
    for (uint32_t i = 0; i < count; i++)
        if (!hs[i]) return SD_ERR_ARG;
    sd_handle *d = hs[0];
    DeviceGuard dg(d->p.device);
    if (d->T.mode == 6) return update_many_planes(hs, pairs, ns, count);
    const sd_params &P = d->p;
    BatchLayout BL{};
    const bool binnable = batch_layout(d, &BL);
    const uint32_t S_link = BL.S_link, sl = BL.sl;
    const uint32_t max_members = S_link ? 4096u / S_link : 1u;
    const uint64_t chunk = 1ull << d->T.bin_chunk_log2;

    // which links join the batch: device-resident pairs on hs[0]'s device,
    // the same DHLA shape, each handle once; the others update on their own
    std::vector<uint32_t> batch;
    for (uint32_t i = 0; i < count; i++) {
        if (binnable && batch_member(d, hs[i], pairs[i], ns[i], hs, batch)) {
            batch.push_back(i);
        } else {
            const int rc = sd_update(hs[i], pairs[i], ns[i]);
            if (rc != SD_OK) return rc;
        }
    }
    if (batch.empty()) return SD_OK;

    // the rounds' link tables live side by side in one buffer
    uint64_t rounds_upper = 1;
    for (uint32_t q : batch) rounds_upper += (ns[q] + chunk - 1) / chunk;
    const uint64_t need = rounds_upper * std::min<uint64_t>(batch.size(), max_members);
    const int half = d->links_half ^ 1;
    if (d->links_cap < need) {
        SD_CK(d, cudaStreamSynchronize(d->stream));  // earlier batches may still read the tables
        cudaFree(d->links_dev);
        cudaFreeHost(d->links_h);
        d->links_dev = nullptr;
        d->links_h = nullptr;
        d->links_cap = 0;
        SD_CK(d, cudaMalloc(&d->links_dev, 2 * need * sizeof(LinkDesc)));
        SD_CK(d, cudaMallocHost(&d->links_h, 2 * need * sizeof(LinkDesc)));
        d->links_cap = (uint32_t)need;
    } else {
        SD_CK(d, cudaEventSynchronize(d->ev_links[half]));  // the call two back has read this half
    }
    d->links_half = half;
    LinkDesc *const tab_h = d->links_h + (size_t)half * d->links_cap;
    LinkDesc *const tab_d = d->links_dev + (size_t)half * d->links_cap;
    // the members' earlier work comes first, on the driver's stream
    for (uint32_t q : batch) {
        sd_handle *h = hs[q];
        if (h == d || h->stream == d->stream) continue;
        SD_CK(h, cudaEventRecord(h->ev_batch, h->stream));
        SD_CK(d, cudaStreamWaitEvent(d->stream, h->ev_batch, 0));
    }

    const uint32_t TP = d->T.bin_tile_pairs;
    std::vector<uint64_t> done(batch.size(), 0);
    size_t cursor = 0, tab_used = 0;
    for (;;) {
        // the round's members, round-robin among links with pairs left: as
        // many as the bins allow at the largest member share of the round
        // (a share is up to one chunk), at most 4096 slices in all
        std::vector<uint32_t> mem;
        uint64_t max_take = 0;
        for (size_t t = 0; t < batch.size() && mem.size() < max_members; t++) {
            const size_t q = (cursor + t) % batch.size();
            if (done[q] >= ns[batch[q]]) continue;
            const uint64_t take = std::min(chunk, ns[batch[q]] - done[q]);
            const uint64_t mt = std::max(max_take, take);
            const uint64_t bytes = (uint64_t)(mem.size() + 1) * S_link * BL.cap_for(mt) * 4;
            if (!mem.empty() && bytes > BL.bin_bytes) break;
            mem.push_back((uint32_t)q);
            max_take = mt;
        }
        if (mem.empty()) break;
        cursor = (mem.back() + 1) % batch.size();
        const uint64_t budget = chunk;
        LinkDesc *tab = tab_h + tab_used;
        uint64_t tiles = 0;
        for (uint32_t m = 0; m < mem.size(); m++) {
            const uint32_t i = batch[mem[m]];
            const sd_handle *h = hs[i];
            const uint64_t take = std::min(budget, ns[i] - done[mem[m]]);
            LinkDesc &L = tab[m];
            hs[i]->grid_clean = false;
            L.pairs = pairs[i] + 2 * done[mem[m]];
            L.n = take;
            L.grid = h->grid;
            L.tile_start = tiles;
            L.slice0 = m * S_link;
            for (int dd = 0; dd < 2; dd++) {
                L.A0[dd] = h->G.h[dd].A0;
                L.A1[dd] = h->G.h[dd].A1;
                L.B1[dd] = h->G.h[dd].B1;
            }
            tiles += (take + TP - 1) / TP;
            done[mem[m]] += take;
        }
        if (tab_used + mem.size() > d->links_cap) return d->fail(SD_ERR_ARG, "sd_update_many: link table overflow");
        SD_CK(d, cudaMemcpyAsync(tab_d + tab_used, tab, mem.size() * sizeof(LinkDesc), cudaMemcpyHostToDevice,
                                 d->stream));
        BinArgs B;
        std::memset(&B, 0, sizeof B);
        B.S = (uint32_t)mem.size() * S_link;
        B.slice_log2 = sl;
        B.cap = (uint32_t)BL.cap_for(max_take);
        B.tile_pairs = TP;
        B.total_words = (uint64_t)P.dirs * d->G.dir_words;  // words of one link's DHLA
        const int rc = ensure_bin_mem(d, B);
        if (rc != SD_OK) return rc;
        SD_CK(d, launch_binned_links(tab_d + tab_used, (uint32_t)mem.size(), tiles, S_link, d->G, d->bin,
                                     d->num_sms, d->stream));
        launched(2);
        tab_used += mem.size();
    }
    SD_CK(d, cudaEventRecord(d->ev_links[half], d->stream));
    // later work on each member waits for the batch
    SD_CK(d, cudaEventRecord(d->ev_batch, d->stream));
    for (uint32_t q : batch) {
        sd_handle *h = hs[q];
        h->n_pairs += ns[q];
        if (h == d || h->stream == d->stream) continue;
        SD_CK(h, cudaStreamWaitEvent(h->stream, d->ev_batch, 0));
    }
    return SD_OK;
}

int sd_sync(sd_handle *h) {
    if (!h) return SD_ERR_ARG;
    DeviceGuard dg(h->p.device);
    SD_CK(h, cudaStreamSynchronize(h->stream));
    return SD_OK;
}

// Host wall-clock of the close phases, printed to stderr when the
// environment variable SD_TRACE is set (diagnostics; no effect on results).
struct CloseTrace {
    bool on = std::getenv("SD_TRACE") != nullptr;
    std::chrono::steady_clock::time_point t0 = std::chrono::steady_clock::now(), last = t0;
    double ph[6] = {0, 0, 0, 0, 0, 0};
    void mark(int i) {
        if (!on) return;
        const auto now = std::chrono::steady_clock::now();
        ph[i] += std::chrono::duration<double, std::micro>(now - last).count();
        last = now;
    }
    const char *what = "sd_close_window";
    ~CloseTrace() {
        if (on)
            std::fprintf(stderr, "%s us: stats %.1f restore %.1f bigsort %.1f report+reset %.1f total %.1f\n", what,
                         ph[0], ph[1], ph[2], ph[3],
                         std::chrono::duration<double, std::micro>(std::chrono::steady_clock::now() - t0).count());
    }
};

// The window close in four phases, so that many handles can overlap their
// GPU work and share host synchronisations (sd_close_many).  Each phase only
// queues work on the handle's stream; the caller synchronises the stream
// between phases.
//   A: hot estimators and row statistics (Algorithm 2, first loop; §4.2)
//   B: host decisions (psi, szmax, caps), then restore K, estimate SZ,
//      order small hit lists (Algorithm 2 / Algorithms 3-4, §4.2)
//   C: order the large hit lists
//   D: build the report (Eq. 4), clear the DHLA for the next window
static int close_phase_a(sd_handle *h, sd_report *out) {
    std::memset(out, 0, sizeof *out);
    std::memset(&h->cs, 0, sizeof h->cs);
    h->report.clear();
    h->last_ncand[0] = h->last_ncand[1] = 0;
    if (h->planes_dirty && fold_stats_fit(h->G)) {
        // the fold writes the row statistics as it goes
        const FoldJob job{h->grid, h->planes, h->grid_clean ? 1u : 0u, h->zhot, h->st_d, h->hotmap};
        SD_CK(h, launch_plane_fold(job, nullptr, 1, h->G, h->pa.ps, h->num_sms, h->stream));
        launched(1);
        h->planes_dirty = false;
        h->grid_clean = false;
    } else {
        const int frc = fold_planes(h);
        if (frc != SD_OK) return frc;
        SD_CK(h, launch_row_stats(h->grid, h->G, h->zhot, h->hotmap, h->st_d, h->num_sms, h->stream));
        launched(1);
    }
    SD_CK(h, launch_compact(h->hotmap, h->G, h->he, 2, h->stream));
    launched(1);
    SD_CK(h, cudaMemcpyAsync(h->st_h, h->st_d, sizeof(StatBlock), cudaMemcpyDeviceToHost, h->stream));
    return SD_OK;
}

// Host part of phase B: psi, szmax and the work caps per direction, from the
// row statistics in h->st_h; fills h->cs.A.  False when no direction runs.
static bool close_decide(sd_handle *h, sd_report *out) {
    const Geometry &G = h->G;
    CloseState &c = h->cs;
    RestoreArgs &A = c.A;
    for (uint32_t d = 0; d < G.dirs; d++) {
        for (uint32_t i = 0; i < G.r; i++) {
            out->zr[d][i] = h->st_h->zr[d][i];
            out->n_hot[d][i] = h->st_h->nhot[d][i];
        }
        c.psi[d] = psi_of(G.g, G.r, G.k, h->st_h->zr[d]);
        out->psi[d] = c.psi[d];
        if (c.psi[d] < 0.0) {
            c.flags |= SD_FLAG_SATURATED << (8 * d);
            continue;
        }
        const int szmax = szmax_of(G.g, G.r, c.psi[d], h->p.theta);
        out->szmax[d] = szmax < 0 ? 0 : (uint32_t)szmax;
        const uint64_t n0 = h->st_h->nhot[d][0], n1 = h->st_h->nhot[d][1];
        // the restore work bound: |HE(0)| 2^(32-k) keys have a hot DH_0, a
        // superset of K that bounds both restores' work; the staged join
        // also bounds its first-stage tuples |HE(0)||HE(1)||HE(2)|
        bool over = (n0 << (32u - G.k)) > h->pair_cap;
        if (h->T.restore == 1) {
            const uint64_t n2 = h->st_h->nhot[d][2];
            over = over || (n2 && n0 * n1 > h->pair_cap / n2);
        }
        if (over) {
            c.flags |= SD_FLAG_OVERLOAD_PAIRS << (8 * d);
            continue;
        }
        A.run[d] = 1;
        A.n0[d] = (uint32_t)n0;
        A.n1[d] = (uint32_t)n1;
        A.szmax[d] = szmax;
    }
    A.grid = h->grid;
    A.he = h->he;
    A.hotmap = h->hotmap;
    A.cand = h->cand;
    A.hits = h->hits;
    A.stats = h->st_d;
    A.cand_cap = h->cand_cap;
    A.hits_cap = h->hits_cap;
    return A.run[0] || A.run[1];
}

static int close_phase_b(sd_handle *h, sd_report *out) {
    if (!close_decide(h, out)) return SD_OK;
    const Geometry &G = h->G;
    RestoreArgs &A = h->cs.A;
    if (h->T.restore == 1) {
        if (!h->jsub) {
            h->join_cap = 4 * h->cand_cap;
            SD_CK(h, cudaMalloc(&h->he_all, ((uint64_t)G.dirs * G.r << G.k) * 4));
            SD_CK(h, cudaMalloc(&h->jsub, 2 * G.dirs * h->join_cap * 8));
        }
        JoinArgs J;
        std::memset(&J, 0, sizeof J);
        J.he = h->he_all;
        J.sub[0] = h->jsub;
        J.sub[1] = h->jsub + G.dirs * h->join_cap;
        J.cap = h->join_cap;
        J.cand = h->cand;
        J.cand_cap = h->cand_cap;
        J.stats = h->st_d;
        for (uint32_t d = 0; d < G.dirs; d++) {
            J.run[d] = A.run[d];
            for (uint32_t i = 0; i < G.r; i++) J.n[d][i] = h->st_h->nhot[d][i];
        }
        SD_CK(h, launch_compact(h->hotmap, G, h->he_all, G.r, h->stream));
        SD_CK(h, launch_join(G, J, h->num_sms, h->stream));
        launched(1 + (G.r - 2));
    } else {
        SD_CK(h, launch_restore(G, A, h->num_sms, h->stream));
        launched(((A.run[0] && A.n0[0] && A.n1[0]) || (A.run[1] && A.n0[1] && A.n1[1])) ? 1 : 0);
    }
    SD_CK(h, launch_estimate(G, A, h->num_sms, h->stream));
    SD_CK(h, launch_sort_small(h->hits, h->hits_cap, h->st_d, A.run, G.dirs, h->stream));
    launched(2);
    SD_CK(h, cudaMemcpyAsync(h->st_h, h->st_d, sizeof(StatBlock), cudaMemcpyDeviceToHost, h->stream));
    for (uint32_t d = 0; d < G.dirs; d++)
        if (A.run[d])
            SD_CK(h, cudaMemcpyAsync(h->hits_h + (uint64_t)d * kSortSmall, h->hits + (uint64_t)d * h->hits_cap,
                                     std::min<uint64_t>(kSortSmall, h->hits_cap) * 8, cudaMemcpyDeviceToHost,
                                     h->stream));
    return SD_OK;
}

// Returns SD_OK; sets *need_sync when large sorts were queued.
static int close_phase_c(sd_handle *h, sd_report *out, bool *need_sync) {
    CloseState &c = h->cs;
    *need_sync = false;
    h->ss_check[0] = h->ss_check[1] = false;
    for (uint32_t d = 0; d < h->G.dirs; d++) {
        if (!c.A.run[d]) continue;
        const uint64_t nk = h->st_h->ncand[d];
        out->n_cand[d] = nk;
        h->last_ncand[d] = nk;
        bool join_full = false;  // a staged-join list that overflowed its buffer: K is incomplete
        if (h->T.restore == 1)
            for (uint32_t i = 2; i + 1 < h->G.r; i++) join_full |= h->st_h->jcount[d][i] > h->join_cap;
        if (nk > h->cand_cap || join_full) {
            // the restore stopped once K passed its capacity: |K| is only
            // known to exceed it
            out->n_cand[d] = h->cand_cap + 1;
            h->last_ncand[d] = h->cand_cap + 1;
            c.flags |= SD_FLAG_OVERLOAD_CANDS << (8 * d);
            continue;
        }
        c.nh[d] = h->st_h->nhits[d];
        c.keys[d] = h->hits_h + (uint64_t)d * kSortSmall;
        if (!h->st_h->big_sort[d]) continue;
        unsigned long long *sorted = nullptr;
        uint32_t *overflow = nullptr;
        int nl = 0;
        if (!h->ss_d) {
            SD_CK(h, cudaMalloc(&h->ss_d, 2 * kSampleScratchBytes));
            SD_CK(h, cudaMallocHost(&h->ss_flag_h, 2 * sizeof(uint32_t)));
        }
        SD_CK(h, launch_sort_big(h->hits + (uint64_t)d * h->hits_cap, h->hits_tmp + (uint64_t)d * h->hits_cap,
                                 c.nh[d], static_cast<char *>(h->ss_d) + d * kSampleScratchBytes, h->num_sms,
                                 h->stream, &sorted, &nl, &overflow));
        launched(nl);
        if (!h->big_h) SD_CK(h, cudaMallocHost(&h->big_h, (uint64_t)2 * h->hits_cap * 8));
        unsigned long long *dst = h->big_h + (uint64_t)d * h->hits_cap;
        SD_CK(h, cudaMemcpyAsync(dst, sorted, c.nh[d] * 8, cudaMemcpyDeviceToHost, h->stream));
        h->ss_check[d] = overflow != nullptr;
        if (overflow)
            SD_CK(h, cudaMemcpyAsync(h->ss_flag_h + d, overflow, 4, cudaMemcpyDeviceToHost, h->stream));
        c.keys[d] = dst;
        *need_sync = true;
    }
    return SD_OK;
}

// A sample sort of phase C that fell short (a bucket beyond one block's
// shared memory): the list, still a permutation of the hits on the device,
// is sorted again by the merge path and read back (after phase C's sync).
static int redo_short_sorts(sd_handle *h) {
    CloseState &c = h->cs;
    for (uint32_t d = 0; d < h->G.dirs; d++) {
        if (!h->ss_check[d]) continue;
        h->ss_check[d] = false;
        if (!h->ss_flag_h[d]) continue;
        unsigned long long *sorted = nullptr;
        uint32_t *overflow = nullptr;
        int nl = 0;
        SD_CK(h, launch_sort_big(h->hits + (uint64_t)d * h->hits_cap, h->hits_tmp + (uint64_t)d * h->hits_cap,
                                 c.nh[d], nullptr, h->num_sms, h->stream, &sorted, &nl, &overflow));
        launched(nl);
        SD_CK(h, cudaMemcpyAsync(h->big_h + (uint64_t)d * h->hits_cap, sorted, c.nh[d] * 8, cudaMemcpyDeviceToHost,
                                 h->stream));
        SD_CK(h, cudaStreamSynchronize(h->stream));
    }
    return SD_OK;
}

static int close_phase_d(sd_handle *h, sd_report *out, bool reset = true) {
    const Geometry &G = h->G;
    CloseState &c = h->cs;
    const int src = redo_short_sorts(h);
    if (src != SD_OK) return src;
    for (uint32_t d = 0; d < G.dirs; d++) {
        if (!c.A.run[d] || !c.keys[d]) continue;
        // Eq. 4 depends on SZ alone within a window: one evaluation per
        // distinct SZ value (hits have SZ <= szmax), bit-identical to
        // evaluating it per hit
        std::vector<double> &tbl = h->est_tbl;
        tbl.assign((size_t)(c.A.szmax[d] >= 0 ? c.A.szmax[d] + 1 : 0), 0.0);
        for (size_t z = 0; z < tbl.size(); z++) tbl[z] = eq4(G.g, G.r, c.psi[d], (uint32_t)z);
        const uint64_t nh = c.nh[d];
        const unsigned long long *keys = c.keys[d];
        const size_t at = h->report.size();
        h->report.grow_to(at + nh);
        sd_hit *out_h = h->report.data() + at;
        const double *t = tbl.data();
        const size_t tn = tbl.size();
        for (uint64_t q = 0; q < nh; q++) {
            const unsigned long long key = keys[q];
            const uint32_t sz = (uint32_t)(key & 0xFFFFFFFFull);
            out_h[q].ip = (uint32_t)(key >> 32);
            out_h[q].sz = sz;
            out_h[q].dir = d;
            out_h[q].reserved = 0;
            out_h[q].est = sz < tn ? t[sz] : eq4(G.g, G.r, c.psi[d], sz);
        }
    }
    h->have_close = true;
    // clear the DHLA and the counters for the next window (stream-ordered;
    // a batched close clears all its handles in one launch instead)
    if (reset) {
        SD_CK(h, launch_reset(h->grid, (uint64_t)G.dirs * G.dir_words, h->st_d, h->num_sms, h->stream));
        launched(1);
        h->grid_clean = !h->planes_dirty;
    }

    uint32_t flags = c.flags;
    out->n_hits_total = h->report.size();
    if (h->report.size() > h->report_cap) {
        for (uint64_t q = h->report_cap; q < h->report.size(); q++)
            flags |= SD_FLAG_REPORT_OVERFLOW << (8 * h->report[q].dir);
        h->report.truncate(h->report_cap);
    }
    out->n_pairs = h->n_pairs;
    h->n_pairs = 0;
    out->zhot = (uint32_t)(h->zhot < 0 ? 0 : h->zhot);
    out->flags = flags;
    out->n_hits = h->report.size();
    out->hits = h->report.empty() ? nullptr : h->report.data();

    const uint32_t any = flags | (flags >> 8);
    if (any & SD_FLAG_SATURATED) return h->fail(SD_ERR_SATURATED, "sd_close_window: a row is saturated (ZR = 0)");
    if (any & (SD_FLAG_OVERLOAD_PAIRS | SD_FLAG_OVERLOAD_CANDS))
        return h->fail(SD_ERR_OVERLOAD, "sd_close_window: restore over its pair or candidate cap");
    if (any & SD_FLAG_REPORT_OVERFLOW)
        return h->fail(SD_ERR_REPORT_OVERFLOW, "sd_close_window: more hits than report_cap");
    return SD_OK;
}

static bool rc_is_error(int rc) { return rc == SD_ERR_ARG || rc == SD_ERR_NOMEM || rc == SD_ERR_CUDA; }

int sd_close_window(sd_handle *h, sd_report *out) {
    NvtxRange nvtx("sd_close_window");
    if (!h || !out) return SD_ERR_ARG;
    DeviceGuard dg(h->p.device);
    // the close runs on the handle's high-priority side stream, after
    // everything queued on its stream, and the stream waits for the close
    SD_CK(h, cudaEventRecord(h->ev_batch, h->stream));
    SD_CK(h, cudaStreamWaitEvent(h->copy_stream, h->ev_batch, 0));
    std::swap(h->stream, h->copy_stream);
    struct Rejoin {
        sd_handle *h;
        ~Rejoin() {
            std::swap(h->stream, h->copy_stream);
            cudaEventRecord(h->ev_batch, h->copy_stream);
            cudaStreamWaitEvent(h->stream, h->ev_batch, 0);
        }
    } rejoin{h};
    CloseTrace trace;
    int rc = close_phase_a(h, out);
    if (rc != SD_OK) return rc;
    SD_CK(h, cudaStreamSynchronize(h->stream));
    trace.mark(0);
    rc = close_phase_b(h, out);
    if (rc != SD_OK) return rc;
    SD_CK(h, cudaStreamSynchronize(h->stream));
    trace.mark(1);
    bool big = false;
    rc = close_phase_c(h, out, &big);
    if (rc != SD_OK) return rc;
    if (big) SD_CK(h, cudaStreamSynchronize(h->stream));
    trace.mark(2);
    rc = close_phase_d(h, out);
    trace.mark(3);
    return rc;
}

// sd_close_many for handles of one DHLA shape on one device that use the
// default restore: every phase is one launch (or a few) over all the
// handles, on hs[0]'s stream, with one host synchronisation per phase; the
// host decisions per handle are the same functions as for one window.
static bool batchable(sd_handle *const *hs, uint32_t count) {
    if (count < 2) return false;
    const sd_params &P = hs[0]->p;
    for (uint32_t i = 0; i < count; i++) {
        const sd_handle *h = hs[i];
        if (h->p.device != P.device || h->p.g != P.g || h->p.r != P.r || h->p.k != P.k ||
            h->p.alpha != P.alpha || h->p.dirs != P.dirs || h->T.restore != 0)
            return false;
    }
    return true;
}

static int close_many_batched(sd_handle *const *hs, uint32_t count, sd_report *outs, int *rcs) {
    CloseTrace tr;
    tr.what = "sd_close_many (batched)";
    sd_handle *d = hs[0];
    DeviceGuard dg(d->p.device);
    const Geometry &G = d->G;
    cudaStream_t s = d->stream;
    if (d->cj_cap < count) {
        SD_CK(d, cudaStreamSynchronize(s));
        cudaFree(d->cj_d);
        cudaFreeHost(d->cj_h);
        cudaFree(d->cb_st_d);
        cudaFreeHost(d->cb_st_h);
        cudaFree(d->cb_hits_d);
        cudaFreeHost(d->cb_hits_h);
        cudaFree(d->cb_base_d);
        cudaFreeHost(d->cb_base_h);
        cudaFree(d->fj_d);
        cudaFreeHost(d->fj_h);
        d->fj_d = d->fj_h = nullptr;
        d->cj_d = d->cj_h = nullptr;
        d->cb_st_d = d->cb_st_h = nullptr;
        d->cb_hits_d = d->cb_hits_h = nullptr;
        d->cb_base_d = d->cb_base_h = nullptr;
        d->cj_cap = 0;
        SD_CK(d, cudaMalloc(&d->cj_d, count * sizeof(CloseJob)));
        SD_CK(d, cudaMallocHost(&d->cj_h, count * sizeof(CloseJob)));
        SD_CK(d, cudaMalloc(&d->cb_st_d, count * sizeof(StatBlock)));
        SD_CK(d, cudaMallocHost(&d->cb_st_h, count * sizeof(StatBlock)));
        SD_CK(d, cudaMalloc(&d->cb_hits_d, (uint64_t)count * 2 * kSortSmall * 8));
        SD_CK(d, cudaMallocHost(&d->cb_hits_h, (uint64_t)count * 2 * kSortSmall * 8));
        // tile offsets (device + host) and candidate offsets (device), 2 count + 1 each
        SD_CK(d, cudaMalloc(&d->cb_base_d, (uint64_t)2 * (2 * count + 1) * 8));
        SD_CK(d, cudaMallocHost(&d->cb_base_h, (uint64_t)(2 * count + 1) * 8));
        SD_CK(d, cudaMalloc(&d->fj_d, count * sizeof(FoldJob)));
        SD_CK(d, cudaMallocHost(&d->fj_h, count * sizeof(FoldJob)));
        d->cj_cap = count;
    }
    // every member's queued work comes first, on the driver's stream
    for (uint32_t i = 1; i < count; i++) {
        sd_handle *h = hs[i];
        if (h->stream == s) continue;
        SD_CK(h, cudaEventRecord(h->ev_batch, h->stream));
        SD_CK(d, cudaStreamWaitEvent(s, h->ev_batch, 0));
    }
    // phase A: row statistics and HE(0), HE(1) of every window (pending
    // plane-binned updates folded into each DHLA first, all in one launch
    // on the driver's stream, which is ordered after every member's work)
    // (with the row statistics where the shape allows: those members skip
    // k_row_stats_many)
    uint32_t nfold = 0;
    const bool fold_stats = fold_stats_fit(G);
    std::vector<char> folded(count, 0);
    for (uint32_t i = 0; i < count; i++) {
        sd_handle *h = hs[i];
        if (!h->planes_dirty) continue;
        d->fj_h[nfold++] = FoldJob{h->grid, h->planes, h->grid_clean ? 1u : 0u, h->zhot,
                                   fold_stats ? h->st_d : nullptr, fold_stats ? h->hotmap : nullptr};
        folded[i] = fold_stats;
        h->planes_dirty = false;
        h->grid_clean = false;
    }
    if (nfold) {
        SD_CK(d, cudaMemcpyAsync(d->fj_d, d->fj_h, nfold * sizeof(FoldJob), cudaMemcpyHostToDevice, s));
        SD_CK(d, launch_plane_fold(d->fj_h[0], d->fj_d, nfold, G, plane_words(G), d->num_sms, s));
        launched(1);
    }
    for (uint32_t i = 0; i < count; i++) {
        sd_handle *h = hs[i];
        std::memset(&outs[i], 0, sizeof outs[i]);
        std::memset(&h->cs, 0, sizeof h->cs);
        h->report.clear();
        h->last_ncand[0] = h->last_ncand[1] = 0;
        CloseJob &j = d->cj_h[i];
        std::memset(&j, 0, sizeof j);
        j.G = h->G;
        j.A.grid = h->grid;
        j.A.he = h->he;
        j.A.hotmap = h->hotmap;
        j.A.stats = h->st_d;
        j.zhot = h->zhot;
        j.stats_done = folded[i];
        rcs[i] = SD_OK;
    }
    SD_CK(d, cudaMemcpyAsync(d->cj_d, d->cj_h, count * sizeof(CloseJob), cudaMemcpyHostToDevice, s));
    SD_CK(d, launch_stats_many(d->cj_d, count, G, d->num_sms, s));
    SD_CK(d, launch_gather_many(d->cj_d, count, d->cb_st_d, d->cb_hits_d, s));
    launched(3);
    SD_CK(d, cudaMemcpyAsync(d->cb_st_h, d->cb_st_d, count * sizeof(StatBlock), cudaMemcpyDeviceToHost, s));
    SD_CK(d, cudaStreamSynchronize(s));
    tr.mark(0);
    // phase B: host decisions per window, then restore, estimate and the
    // small sorts of all of them
    bool any = false;
    for (uint32_t i = 0; i < count; i++) {
        sd_handle *h = hs[i];
        *h->st_h = d->cb_st_h[i];
        const bool run = close_decide(h, &outs[i]);
        CloseJob &j = d->cj_h[i];
        j.A = h->cs.A;
        if (run) prepare_restore(G, j.A, d->num_sms, 1);
        h->cs.A = j.A;
        any = any || run;
    }
    if (any) {
        SD_CK(d, cudaMemcpyAsync(d->cj_d, d->cj_h, count * sizeof(CloseJob), cudaMemcpyHostToDevice, s));
        int nl = 0;
        SD_CK(d, launch_restore_many(d->cj_d, d->cj_h, count, d->cb_base_d, d->cb_base_h,
                                     d->cb_base_d + (2 * count + 1), d->num_sms, s, &nl));
        SD_CK(d, launch_gather_many(d->cj_d, count, d->cb_st_d, d->cb_hits_d, s));
        launched(nl + 1);
        SD_CK(d, cudaMemcpyAsync(d->cb_st_h, d->cb_st_d, count * sizeof(StatBlock), cudaMemcpyDeviceToHost, s));
        SD_CK(d, cudaMemcpyAsync(d->cb_hits_h, d->cb_hits_d, (uint64_t)count * 2 * kSortSmall * 8,
                                 cudaMemcpyDeviceToHost, s));
        SD_CK(d, cudaStreamSynchronize(s));
    }
    tr.mark(1);
    // phase C: caps, and the rare hit lists too long for one block's sort
    std::vector<char> big(count, 0);
    bool any_big = false;
    for (uint32_t i = 0; i < count; i++) {
        sd_handle *h = hs[i];
        if (!any) continue;
        *h->st_h = d->cb_st_h[i];
        bool b = false;
        rcs[i] = close_phase_c(h, &outs[i], &b);
        for (uint32_t dd = 0; dd < G.dirs; dd++)
            if (h->cs.keys[dd] == h->hits_h + (uint64_t)dd * kSortSmall)
                h->cs.keys[dd] = d->cb_hits_h + ((uint64_t)i * 2 + dd) * kSortSmall;
        big[i] = b;
        any_big = any_big || b;
    }
    if (any_big)
        for (uint32_t i = 0; i < count; i++)
            if (big[i]) SD_CK(hs[i], cudaStreamSynchronize(hs[i]->stream));
    tr.mark(2);
    // phase D: the reports, then one reset of every DHLA
    for (uint32_t i = 0; i < count; i++)
        if (rcs[i] == SD_OK) rcs[i] = close_phase_d(hs[i], &outs[i], false);
    SD_CK(d, launch_reset_many(d->cj_d, count, G, d->num_sms, s));
    launched(1);
    for (uint32_t i = 0; i < count; i++) hs[i]->grid_clean = !hs[i]->planes_dirty;
    tr.mark(3);
    // each member's later work waits for the batch
    SD_CK(d, cudaEventRecord(d->ev_batch, s));
    for (uint32_t i = 1; i < count; i++) {
        sd_handle *h = hs[i];
        if (h->stream == s) continue;
        SD_CK(h, cudaStreamWaitEvent(h->stream, d->ev_batch, 0));
    }
    for (uint32_t i = 0; i < count; i++)
        if (rc_is_error(rcs[i])) return rcs[i];
    return SD_OK;
}

int sd_close_many(sd_handle *const *hs, uint32_t count, sd_report *outs, int *rcs) {
    NvtxRange nvtx("sd_close_many");
    if (!hs || !outs || !rcs) return count ? SD_ERR_ARG : SD_OK;
    for (uint32_t i = 0; i < count; i++)
        if (!hs[i]) return SD_ERR_ARG;
    {
        std::vector<sd_handle *> sorted(hs, hs + count);
        std::sort(sorted.begin(), sorted.end());
        if (std::adjacent_find(sorted.begin(), sorted.end()) != sorted.end()) return SD_ERR_ARG;
    }
    if (batchable(hs, count)) return close_many_batched(hs, count, outs, rcs);
    // Each handle's close runs on its side stream (ordered after everything
    // queued on its stream so far, and its stream waits for the close), so
    // the closes of handles that share one stream still overlap on the GPU.
    const bool side = count > 1;
    if (side) {
        for (uint32_t i = 0; i < count; i++) {
            sd_handle *h = hs[i];
            DeviceGuard dg(h->p.device);
            SD_CK(h, cudaEventRecord(h->ev_batch, h->stream));
            SD_CK(h, cudaStreamWaitEvent(h->copy_stream, h->ev_batch, 0));
        }
        for (uint32_t i = 0; i < count; i++) std::swap(hs[i]->stream, hs[i]->copy_stream);
    }
    struct Unswap {
        sd_handle *const *hs;
        uint32_t count;
        bool on;
        ~Unswap() {
            if (!on) return;
            for (uint32_t i = 0; i < count; i++) {
                sd_handle *h = hs[i];
                std::swap(h->stream, h->copy_stream);
                DeviceGuard dg(h->p.device);
                cudaEventRecord(h->ev_batch, h->copy_stream);
                cudaStreamWaitEvent(h->stream, h->ev_batch, 0);
            }
        }
    } unswap{hs, count, side};
    std::vector<char> live(count, 1);
    auto step = [&](auto &&phase) {
        for (uint32_t i = 0; i < count; i++) {
            if (!live[i]) continue;
            DeviceGuard dg(hs[i]->p.device);
            rcs[i] = phase(hs[i], &outs[i], i);
            if (rcs[i] != SD_OK) live[i] = 0;
        }
    };
    auto sync = [&](const std::vector<char> &which) {
        for (uint32_t i = 0; i < count; i++) {
            if (!live[i] || !which[i]) continue;
            DeviceGuard dg(hs[i]->p.device);
            const cudaError_t e = cudaStreamSynchronize(hs[i]->stream);
            if (e != cudaSuccess) {
                rcs[i] = hs[i]->fail(SD_ERR_CUDA, "sd_close_many: %s", cudaGetErrorString(e));
                live[i] = 0;
            }
        }
    };
    std::vector<char> all(count, 1), big(count, 0);
    for (uint32_t i = 0; i < count; i++) rcs[i] = SD_OK;
    step([](sd_handle *h, sd_report *o, uint32_t) { return close_phase_a(h, o); });
    sync(all);
    step([](sd_handle *h, sd_report *o, uint32_t) { return close_phase_b(h, o); });
    sync(all);
    step([&](sd_handle *h, sd_report *o, uint32_t i) {
        bool b = false;
        const int rc = close_phase_c(h, o, &b);
        big[i] = b;
        return rc;
    });
    sync(big);
    for (uint32_t i = 0; i < count; i++) {
        if (!live[i]) continue;
        DeviceGuard dg(hs[i]->p.device);
        rcs[i] = close_phase_d(hs[i], &outs[i]);
    }
    for (uint32_t i = 0; i < count; i++)
        if (rc_is_error(rcs[i])) return rcs[i];
    return SD_OK;
}

int sd_destroy(sd_handle *h) {
    if (!h) return SD_OK;
    {
        DeviceGuard dg(h->p.device);
        release(h);
    }
    delete h;
    return SD_OK;
}

const char *sd_last_error(const sd_handle *h) {
    return h ? h->err.c_str() : g_create_error.c_str();
}

int sd_get_grid(sd_handle *h, uint32_t dir, uint32_t *host_dst) {
    if (!h || !host_dst || dir >= h->G.dirs) return SD_ERR_ARG;
    DeviceGuard dg(h->p.device);
    const int frc = fold_planes(h);
    if (frc != SD_OK) return frc;
    SD_CK(h, cudaMemcpyAsync(host_dst, h->grid + (uint64_t)dir * h->G.dir_words, h->G.dir_words * 4,
                             cudaMemcpyDeviceToHost, h->stream));
    SD_CK(h, cudaStreamSynchronize(h->stream));
    return SD_OK;
}

int sd_set_grid(sd_handle *h, uint32_t dir, const uint32_t *host_src) {
    if (!h || !host_src || dir >= h->G.dirs) return SD_ERR_ARG;
    DeviceGuard dg(h->p.device);
    const int frc = fold_planes(h);  // pending bits of the other direction stay
    if (frc != SD_OK) return frc;
    h->grid_clean = false;
    SD_CK(h, cudaMemcpyAsync(h->grid + (uint64_t)dir * h->G.dir_words, host_src, h->G.dir_words * 4,
                             cudaMemcpyHostToDevice, h->stream));
    SD_CK(h, cudaStreamSynchronize(h->stream));
    return SD_OK;
}

int sd_get_hot(sd_handle *h, uint32_t dir, uint32_t row, uint32_t *host_bitmap) {
    if (!h || !host_bitmap || dir >= h->G.dirs || row >= h->G.r) return SD_ERR_ARG;
    if (!h->have_close) return h->fail(SD_ERR_ARG, "sd_get_hot: no window has been closed yet");
    DeviceGuard dg(h->p.device);
    const uint64_t nw = ((uint64_t)1 << h->G.k) >> 5;
    SD_CK(h, cudaMemcpyAsync(host_bitmap, h->hotmap + ((uint64_t)dir * h->G.r + row) * nw, nw * 4,
                             cudaMemcpyDeviceToHost, h->stream));
    SD_CK(h, cudaStreamSynchronize(h->stream));
    return SD_OK;
}

int64_t sd_get_candidates(sd_handle *h, uint32_t dir, uint32_t *host_dst, uint64_t cap) {
    if (!h || dir >= h->G.dirs || (cap && !host_dst)) return SD_ERR_ARG;
    if (!h->have_close) return h->fail(SD_ERR_ARG, "sd_get_candidates: no window has been closed yet");
    DeviceGuard dg(h->p.device);
    const uint64_t nk = h->last_ncand[dir];
    const uint64_t m = std::min(std::min(nk, h->cand_cap), cap);
    if (m) {
        SD_CK(h, cudaMemcpyAsync(host_dst, h->cand + (uint64_t)dir * h->cand_cap, m * 4, cudaMemcpyDeviceToHost,
                                 h->stream));
        SD_CK(h, cudaStreamSynchronize(h->stream));
    }
    return (int64_t)nk;
}

int sd_merge(sd_handle *dst, sd_handle *src) {
    NvtxRange nvtx("sd_merge");
    if (!dst || !src || dst == src) return SD_ERR_ARG;
    const sd_params &a = dst->p, &b = src->p;
    if (a.g != b.g || a.r != b.r || a.k != b.k || a.alpha != b.alpha || a.seed != b.seed || a.dirs != b.dirs ||
        a.device != b.device)
        return dst->fail(SD_ERR_ARG, "sd_merge: handles differ in shape, seed or device");
    DeviceGuard dg(a.device);
    int frc = fold_planes(src);
    if (frc == SD_OK) frc = fold_planes(dst);
    if (frc != SD_OK) return frc;
    dst->grid_clean = false;
    cudaEvent_t ev;
    SD_CK(dst, cudaEventCreateWithFlags(&ev, cudaEventDisableTiming));
    cudaError_t e = cudaEventRecord(ev, src->stream);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(dst->stream, ev, 0);
    if (e == cudaSuccess) {
        e = launch_merge(dst->grid, src->grid, (uint64_t)a.dirs * dst->G.dir_words, dst->num_sms, dst->stream);
        if (e == cudaSuccess) launched(1);
    }
    if (e == cudaSuccess) e = cudaEventRecord(ev, dst->stream);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(src->stream, ev, 0);  // src may not change until merged
    cudaEventDestroy(ev);
    if (e != cudaSuccess) return dst->fail(SD_ERR_CUDA, "sd_merge: %s", cudaGetErrorString(e));
    dst->n_pairs += src->n_pairs;
    return SD_OK;
}

// Is p 16-byte aligned device (or managed) memory of `dev`?
static bool device_buffer(const void *p, int dev) {
    if (!p || ((uintptr_t)p & 15u)) return false;
    cudaPointerAttributes a;
    if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return (a.type == cudaMemoryTypeDevice && a.device == dev) || a.type == cudaMemoryTypeManaged;
}

int sd_export_grid(sd_handle *h, uint32_t *dst) {
    NvtxRange nvtx("sd_export_grid");
    if (!h) return SD_ERR_ARG;
    if (!device_buffer(dst, h->p.device))
        return h->fail(SD_ERR_ARG, "sd_export_grid: dst is not 16-byte aligned memory of device %d", h->p.device);
    DeviceGuard dg(h->p.device);
    const int frc = fold_planes(h);
    if (frc != SD_OK) return frc;
    SD_CK(h, cudaMemcpyAsync(dst, h->grid, (uint64_t)h->G.dirs * h->G.dir_words * 4, cudaMemcpyDeviceToDevice,
                             h->stream));
    return SD_OK;
}

int sd_or_grid(sd_handle *h, const uint32_t *src) {
    NvtxRange nvtx("sd_or_grid");
    if (!h) return SD_ERR_ARG;
    if (!device_buffer(src, h->p.device))
        return h->fail(SD_ERR_ARG, "sd_or_grid: src is not 16-byte aligned memory of device %d", h->p.device);
    DeviceGuard dg(h->p.device);
    const int frc = fold_planes(h);
    if (frc != SD_OK) return frc;
    h->grid_clean = false;
    SD_CK(h, launch_merge(h->grid, src, (uint64_t)h->G.dirs * h->G.dir_words, h->num_sms, h->stream));
    launched(1);
    return SD_OK;
}

int sd_or_words(uint32_t *dst, const uint32_t *src, uint64_t words, uint32_t count, void *cuda_stream) {
    NvtxRange nvtx("sd_or_words");
    if (!dst || !src || !count || (words & 3u)) return SD_ERR_ARG;
    if (!words) return SD_OK;
    int dev = -1;
    if (cudaGetDevice(&dev) != cudaSuccess) return SD_ERR_CUDA;
    if (!device_buffer(dst, dev) || !device_buffer(src, dev)) return SD_ERR_ARG;
    int num_sms = 0;
    if (cudaDeviceGetAttribute(&num_sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return SD_ERR_CUDA;
    if (launch_or_words(dst, src, words, count, num_sms, (cudaStream_t)cuda_stream) != cudaSuccess)
        return SD_ERR_CUDA;
    launched(1);
    return SD_OK;
}

int sd_partition_pairs(sd_handle *h, uint32_t dir, const uint32_t *pairs, uint64_t n, uint32_t parts,
                       uint32_t *out, uint64_t *counts) {
    NvtxRange nvtx("sd_partition_pairs");
    if (!h || !counts || (n && (!pairs || !out))) return SD_ERR_ARG;
    if (dir > 1 || parts < 1 || parts > 1024 || (parts & (parts - 1)))
        return h->fail(SD_ERR_ARG, "sd_partition_pairs: dir must be 0 or 1 and parts a power of two up to 1024");
    if (n == 0) {
        for (uint32_t q = 0; q < parts; q++) counts[q] = 0;
        return SD_OK;
    }
    DeviceGuard dg(h->p.device);
    auto on_device = [&](const void *ptr) {
        if (!ptr || ((uintptr_t)ptr & 3u)) return false;
        cudaPointerAttributes a;
        if (cudaPointerGetAttributes(&a, ptr) != cudaSuccess) {
            cudaGetLastError();
            return false;
        }
        return (a.type == cudaMemoryTypeDevice && a.device == h->p.device) || a.type == cudaMemoryTypeManaged;
    };
    if (!on_device(pairs) || !on_device(out))
        return h->fail(SD_ERR_ARG, "sd_partition_pairs: pairs and out must be 4-byte aligned memory of device %d",
                       h->p.device);
    if (!h->part_d) {
        SD_CK(h, cudaMalloc(&h->part_d, 2 * 1024 * sizeof(unsigned long long)));
        SD_CK(h, cudaMallocHost(&h->part_h, 1024 * sizeof(unsigned long long)));
    }
    SD_CK(h, cudaMemsetAsync(h->part_d, 0, parts * sizeof(unsigned long long), h->stream));
    SD_CK(h, launch_partition(pairs, n, dir, parts, h->part_d, nullptr, nullptr, h->num_sms, h->stream, false));
    SD_CK(h, cudaMemcpyAsync(h->part_h, h->part_d, parts * sizeof(unsigned long long), cudaMemcpyDeviceToHost,
                             h->stream));
    SD_CK(h, cudaStreamSynchronize(h->stream));
    unsigned long long run = 0;
    for (uint32_t q = 0; q < parts; q++) {
        counts[q] = h->part_h[q];
        h->part_h[q] = run;  // cursor of part q: its first slot
        run += counts[q];
    }
    unsigned long long *cursor = h->part_d + 1024;
    SD_CK(h, cudaMemcpyAsync(cursor, h->part_h, parts * sizeof(unsigned long long), cudaMemcpyHostToDevice,
                             h->stream));
    SD_CK(h, launch_partition(pairs, n, dir, parts, nullptr, cursor, out, h->num_sms, h->stream, true));
    launched(2);
    SD_CK(h, cudaStreamSynchronize(h->stream));  // the cursors' host copy is reused by the next call
    return SD_OK;
}

uint64_t sd_kernel_launches(void) { return g_launches.load(std::memory_order_relaxed); }

int sd_get_tuning(const sd_handle *h, sd_tuning *out) {
    if (!h || !out) return SD_ERR_ARG;
    out->mode = h->T.mode;
    out->block_threads = h->T.block_threads;
    out->blocks_per_sm = h->T.blocks_per_sm;
    out->unroll = h->T.unroll;
    out->filter_log2 = h->T.filter_log2;
    out->bin_slice_log2 = h->T.bin_slice_log2;
    out->bin_tile_pairs = h->T.bin_tile_pairs;
    out->bin_chunk_log2 = h->T.bin_chunk_log2;
    out->bin_slack_pct = h->T.bin_slack_pct;
    out->restore = h->T.restore;
    out->bin_batch_mib = h->T.bin_batch_mib;
    out->plane_tile_pairs = h->T.plane_tile_pairs;
    out->plane_round_log2 = h->T.plane_round_log2;
    out->plane_unit_log2 = h->T.plane_unit_log2;
    return SD_OK;
}

int sd_set_tuning(sd_handle *h, const sd_tuning *t) {
    if (!h || !t) return SD_ERR_ARG;
    Tuning T = h->T;
    if (t->mode > 6) return h->fail(SD_ERR_ARG, "sd_set_tuning: mode must be 0..6");
    if (t->mode == 6 && !plane_fits(h->G))
        return h->fail(SD_ERR_ARG, "sd_set_tuning: mode 6 needs one bit plane (r 2^k bits) within %llu KiB",
                       (unsigned long long)(kPlaneSmemMax >> 10));
    T.mode = t->mode;
    if (t->restore > 1) return h->fail(SD_ERR_ARG, "sd_set_tuning: restore must be 0 or 1");
    T.restore = t->restore;
    if (t->block_threads) {
        if (t->block_threads < 64 || t->block_threads > 1024 || (t->block_threads & 31))
            return h->fail(SD_ERR_ARG, "sd_set_tuning: block_threads must be a multiple of 32 in [64, 1024]");
        T.block_threads = t->block_threads;
    }
    if (t->blocks_per_sm) T.blocks_per_sm = t->blocks_per_sm;
    if (t->unroll) {
        if (t->unroll != 1 && t->unroll != 2 && t->unroll != 4)
            return h->fail(SD_ERR_ARG, "sd_set_tuning: unroll must be 1, 2 or 4");
        T.unroll = t->unroll;
    }
    if (t->filter_log2) {
        if (t->filter_log2 < 8 || t->filter_log2 > 14)
            return h->fail(SD_ERR_ARG, "sd_set_tuning: filter_log2 must be in [8, 14]");
        T.filter_log2 = t->filter_log2;
    }
    if (t->bin_slice_log2) {
        if (t->bin_slice_log2 < 10 || t->bin_slice_log2 > 15)
            return h->fail(SD_ERR_ARG, "sd_set_tuning: bin_slice_log2 must be in [10, 15]");
        T.bin_slice_log2 = t->bin_slice_log2;
    }
    if (t->bin_tile_pairs) {
        const uint32_t tp = t->bin_tile_pairs;
        const uint32_t tmax = h->G.dirs * h->G.r > 8 ? 1024u : 2048u;
        if (tp < 64 || tp > tmax || (tp & (tp - 1)))
            return h->fail(SD_ERR_ARG, "sd_set_tuning: bin_tile_pairs must be a power of two in [64, %u]", tmax);
        T.bin_tile_pairs = tp;
    }
    if (t->bin_chunk_log2) {
        if (t->bin_chunk_log2 < 12 || t->bin_chunk_log2 > 28)
            return h->fail(SD_ERR_ARG, "sd_set_tuning: bin_chunk_log2 must be in [12, 28]");
        T.bin_chunk_log2 = t->bin_chunk_log2;
    }
    if (t->bin_slack_pct) T.bin_slack_pct = t->bin_slack_pct == 0xFFFFFFFFu ? 0u : t->bin_slack_pct;
    if (t->bin_batch_mib) {
        if (t->bin_batch_mib > (1u << 20))
            return h->fail(SD_ERR_ARG, "sd_set_tuning: bin_batch_mib must be at most 2^20");
        T.bin_batch_mib = t->bin_batch_mib;
    }
    if (t->plane_tile_pairs) {
        const uint32_t tp = t->plane_tile_pairs;
        if (tp != 1024 && tp != 2048 && tp != 4096 && tp != 8192)
            return h->fail(SD_ERR_ARG, "sd_set_tuning: plane_tile_pairs must be 1024, 2048, 4096 or 8192");
        if (plane_bin_smem_bytes(tp, h->G.dirs, h->G.dirs * h->G.g) > 200 * 1024)
            return h->fail(SD_ERR_ARG, "sd_set_tuning: a binning tile of %u pairs does not fit shared memory", tp);
        T.plane_tile_pairs = tp;
    }
    if (t->plane_round_log2) {
        if (t->plane_round_log2 < 10 || t->plane_round_log2 > 28)
            return h->fail(SD_ERR_ARG, "sd_set_tuning: plane_round_log2 must be in [10, 28]");
        T.plane_round_log2 = t->plane_round_log2;
    }
    if (t->plane_unit_log2) {
        if (t->plane_unit_log2 < 8 || t->plane_unit_log2 > 24)
            return h->fail(SD_ERR_ARG, "sd_set_tuning: plane_unit_log2 must be in [8, 24]");
        T.plane_unit_log2 = t->plane_unit_log2;
    }
    if (T.mode == 5) {
        // the binning tile must fit one block's shared memory
        const uint64_t total = (uint64_t)h->G.dirs * h->G.dir_words;
        uint32_t sl = T.bin_slice_log2;
        while (((total + (1ull << sl) - 1) >> sl) > 4096 && sl < 15) sl++;
        const uint32_t S = (uint32_t)((total + (1ull << sl) - 1) >> sl);
        if (bin_smem_bytes(T.bin_tile_pairs, h->G.dirs * h->G.r, S) > 200 * 1024)
            return h->fail(SD_ERR_ARG, "sd_set_tuning: binning tile too large for shared memory");
    }
    h->T = T;
    return SD_OK;
}

}  // extern "C"
