// sd_fold.cu -- the fold of the plane-binned update's plane-major DHLA copy
// into the estimator-major DHLA (grid |= planes^T, then planes = 0), run
// before anything reads the DHLA: the window close (one launch for every
// handle of a batched close), sd_get_grid, sd_set_grid, sd_merge,
// sd_export_grid and sd_or_grid.
//
// Plane (d, b) holds bit b of every estimator of direction d: its row i
// starts at word i * 2^k/32 and holds estimator c's bit at word c >> 5, bit
// c & 31 (planes are ps words apart).  The DHLA holds estimator c's g bits
// as g/32 consecutive words.  Bit c & 31 of word c >> 5 of row i of plane
// 32 t + j is bit j of word t of estimator c of row i: each 32 x 32 bit block
// (32 planes x 32 estimators) is transposed.
#include "sd_common.cuh"

namespace sd {

// ------------------------------------------------------------------- fold
// One block per tile: TC groups of 32 planes (32 TC consecutive bits of
// every estimator of a row) times W consecutive words of one row of those
// planes (32 W estimators), 32 TC W = 8192 words at most.  The tile is
// copied with coalesced 16-byte asynchronous copies into shared memory (and
// its plane words cleared); each thread (t, w) transposes the 32 x 32 bit
// block of plane group t at word w in registers (32 words of 32 planes ->
// word t of 32 estimators); the results are staged by (t, estimator) and
// each estimator's TC words are written to the DHLA with vector stores.  A
// DHLA known to be all zero ("clean") is written without being read.
//
// Shapes: TC = min(8, g/32), W = min(32, 2^k/32); or, when the fold also
// computes the row statistics, TC = g/32 (8, 16 or 32: the tile holds every
// bit of its estimators) and W = min(2^k/32, 256 / TC).  With statistics each estimator's
// z_0 = g - popcount is tested against zhot, its hot bit goes to the tile's
// W hot bitmap words (written whole), and the tile adds its sum of z_0 and
// its hot count to ZR(i) and |HE(i)| -- what k_row_stats computes.
constexpr uint32_t kFoldThreads = 256;
constexpr uint32_t kFoldTile = 8192;  // words per tile stage (32 TC W)
constexpr size_t kFoldSmem = (size_t)2 * kFoldTile * 4;  // two tile stages

// 32 x 32 bit transpose in registers: afterwards bit j of x[b] is what was
// bit b of x[j] (block swaps of 16, 8, 4, 2 and 1 bits).
__device__ __forceinline__ void transpose32_regs(uint32_t (&x)[32]) {
#pragma unroll
    for (int s = 0; s < 5; s++) {
        const uint32_t j = 16u >> s;
        const uint32_t m = s == 0 ? 0x0000FFFFu : s == 1 ? 0x00FF00FFu : s == 2 ? 0x0F0F0F0Fu
                         : s == 3 ? 0x33333333u : 0x55555555u;
#pragma unroll
        for (uint32_t r = 0; r < 32; r++) {
            if (r & j) continue;
            const uint32_t t = ((x[r] >> j) ^ x[r + j]) & m;
            x[r] ^= t << j;
            x[r + j] ^= t;
        }
    }
}

// Where tile `tile` of a fold lies: its job, direction, row, first plane
// group and first plane word.
struct FoldTile {
    FoldJob job;
    uint32_t d, i, tc0, w0;
};
__device__ __forceinline__ FoldTile fold_tile(uint64_t tile, uint64_t per_job, uint32_t tgroups, uint32_t wgroups,
                                              uint32_t TC, uint32_t W, const Geometry &G, const FoldJob &one,
                                              const FoldJob *jobs) {
    FoldTile f;
    const uint32_t jn = (uint32_t)(tile / per_job);
    f.job = jobs ? jobs[jn] : one;
    uint64_t rest = tile - (uint64_t)jn * per_job;
    f.tc0 = (uint32_t)(rest % tgroups) * TC;
    rest /= tgroups;
    f.w0 = (uint32_t)(rest % wgroups) * W;
    rest /= wgroups;
    f.i = (uint32_t)(rest % G.r);
    f.d = (uint32_t)(rest / G.r);
    return f;
}

// The tile shape of a fold (see above).
__host__ __device__ __forceinline__ void fold_shape(const Geometry &G, bool stats, uint32_t &TC, uint32_t &W) {
    const uint32_t rw = (1u << G.k) >> 5;
    TC = stats ? G.wpc : (G.wpc < 8u ? G.wpc : 8u);
    const uint32_t wmax = stats ? 256u / G.wpc : 32u;
    W = rw < wmax ? rw : wmax;
}

// Folds of several handles of one shape run as one launch (the batched
// close): the tiles of job j follow those of job j - 1.  Two tile stages:
// the next tile's plane words are copied in (cp.async) while the current
// one is transposed; the transposed words are staged in place of the
// current tile's input.
__global__ void __launch_bounds__(kFoldThreads, 3)
k_plane_fold(FoldJob one, const FoldJob *__restrict__ jobs, uint32_t njobs, Geometry G, uint32_t ps,
             uint32_t stats) {
    extern __shared__ uint4 fold_smem[];
    __shared__ uint32_t s_hot[32];
    __shared__ unsigned long long s_zr;
    __shared__ uint32_t s_nhot;
    uint32_t *const stage0 = reinterpret_cast<uint32_t *>(fold_smem);
    const uint32_t wpc = G.wpc;
    uint32_t TC, W;
    fold_shape(G, stats != 0, TC, W);
    const uint32_t rw = (1u << G.k) >> 5;  // plane words per row
    const uint32_t wgroups = rw / W, tgroups = wpc / TC;
    const uint64_t per_job = (uint64_t)G.dirs * G.r * wgroups * tgroups;
    const uint64_t tiles = per_job * njobs;
    const uint32_t W4 = W / 4, rows = 32u * TC;
    const uint32_t tt = threadIdx.x / W, w = threadIdx.x % W;
    const uint32_t lane = threadIdx.x & 31u;
    // a tile's first plane word
    auto plane_base = [&](const FoldTile &f) {
        return f.job.planes + ((uint64_t)f.d * G.g + 32u * f.tc0) * ps + (uint64_t)f.i * rw + f.w0;
    };
    // start copying tile `tile` into stage s (one commit group per call)
    auto issue = [&](uint64_t tile, uint32_t s) {
        if (tile < tiles) {
            const FoldTile f = fold_tile(tile, per_job, tgroups, wgroups, TC, W, G, one, jobs);
            const uint32_t *pb = plane_base(f);
            const uint32_t sa = (uint32_t)__cvta_generic_to_shared(stage0 + s * kFoldTile);
            for (uint32_t q = threadIdx.x; q < rows * W4; q += blockDim.x) {
                const uint32_t row = q / W4, c = q - row * W4;
                asm volatile("cp.async.cg.shared.global [%0], [%1], 16;"
                             ::"r"(sa + 16u * q), "l"(pb + (uint64_t)row * ps + 4u * c)
                             : "memory");
            }
        }
        asm volatile("cp.async.commit_group;" ::: "memory");
    };
    if (threadIdx.x < 32) s_hot[threadIdx.x] = 0;
    if (threadIdx.x == 0) {
        s_zr = 0;
        s_nhot = 0;
    }
    uint32_t cur = 0;
    issue(blockIdx.x, 0);
    for (uint64_t tile = blockIdx.x; tile < tiles; tile += gridDim.x, cur ^= 1u) {
        issue(tile + gridDim.x, cur ^ 1u);
        asm volatile("cp.async.wait_group 1;" ::: "memory");  // this tile's copies are done
        __syncthreads();
        const FoldTile f = fold_tile(tile, per_job, tgroups, wgroups, TC, W, G, one, jobs);
        uint32_t *in = stage0 + cur * kFoldTile;
        // clear the tile's plane words that hold bits
        uint32_t *pb = plane_base(f);
        for (uint32_t q = threadIdx.x; q < rows * W4; q += blockDim.x) {
            const uint4 v = reinterpret_cast<const uint4 *>(in)[q];
            if (v.x | v.y | v.z | v.w) {
                const uint32_t row = q / W4, c = q - row * W4;
                *reinterpret_cast<uint4 *>(pb + (uint64_t)row * ps + 4u * c) = make_uint4(0, 0, 0, 0);
            }
        }
        uint32_t x[32];
        const bool mine = tt < TC;
        if (mine) {
#pragma unroll
            for (uint32_t j = 0; j < 32; j++) x[j] = in[(32u * tt + j) * W + w];
            transpose32_regs(x);
        }
        __syncthreads();  // every read of the input stage is done
        uint32_t *out = in;  // [TC][32 bits][W words]
        if (mine) {
#pragma unroll
            for (uint32_t b = 0; b < 32; b++) out[(tt * 32u + b) * W + w] = x[b];
        }
        __syncthreads();
        // estimator 32 (w0 + w) + b of row i gets words tc0 .. tc0 + TC - 1
        uint32_t *row = f.job.grid + (uint64_t)f.d * G.dir_words + (uint64_t)f.i * G.row_words;
        for (uint32_t e0 = 0; e0 < 32u * W; e0 += blockDim.x) {  // the same trip count for every thread
            const uint32_t e = e0 + threadIdx.x;
            const bool live = e < 32u * W;
            const uint32_t b = e / W, ww = e - b * W;
            uint32_t pop = 0;
            if (live) {
                uint32_t *dst = row + (uint64_t)(32u * (f.w0 + ww) + b) * wpc + f.tc0;
                if ((TC & 3u) == 0) {
                    uint4 *d4 = reinterpret_cast<uint4 *>(dst);
                    for (uint32_t h = 0; h < TC / 4; h++) {
                        uint4 nv = make_uint4(out[((4 * h) * 32u + b) * W + ww], out[((4 * h + 1) * 32u + b) * W + ww],
                                              out[((4 * h + 2) * 32u + b) * W + ww],
                                              out[((4 * h + 3) * 32u + b) * W + ww]);
                        const bool any = (nv.x | nv.y | nv.z | nv.w) != 0;
                        if (!f.job.clean && (any || stats)) {
                            const uint4 c = d4[h];
                            nv.x |= c.x; nv.y |= c.y; nv.z |= c.z; nv.w |= c.w;
                            if (nv.x != c.x || nv.y != c.y || nv.z != c.z || nv.w != c.w) d4[h] = nv;
                        } else if (any) {
                            d4[h] = nv;
                        }
                        pop += __popc(nv.x) + __popc(nv.y) + __popc(nv.z) + __popc(nv.w);
                    }
                } else {
                    for (uint32_t t = 0; t < TC; t++) {
                        uint32_t v = out[(t * 32u + b) * W + ww];
                        if (!f.job.clean && (v || stats)) v |= dst[t];
                        if (out[(t * 32u + b) * W + ww]) dst[t] = v;
                        pop += __popc(v);
                    }
                }
            }
            if (stats) {
                // z_0 of this estimator; hot bits gathered per hot bitmap word
                const uint32_t z0 = G.g - pop;
                const bool hot = live && (int)z0 <= f.job.zhot;
                const unsigned mask = __ballot_sync(0xFFFFFFFFu, hot);
                unsigned long long zs = live ? z0 : 0u;
#pragma unroll
                for (int o = 16; o > 0; o >>= 1) zs += __shfl_xor_sync(0xFFFFFFFFu, zs, o);
                if (lane == 0) {
                    atomicAdd(&s_zr, zs);
                    atomicAdd(&s_nhot, (uint32_t)__popc(mask));
                }
                // the warp's estimators: 32 / W values of b (W < 32) or one
                if (lane < W && live) {
                    const uint32_t b0 = (e - lane) / W;
                    uint32_t c = 0;
                    for (uint32_t qq = 0; qq * W < 32u; qq++) c |= ((mask >> (qq * W + lane)) & 1u) << (b0 + qq);
                    atomicOr(&s_hot[lane], c);
                }
            }
        }
        __syncthreads();  // the stage is refilled two tiles on; the tile's statistics are complete
        if (stats) {
            uint32_t *hm = f.job.hotmap + ((uint64_t)f.d * G.r + f.i) * (rw) + f.w0;
            if (threadIdx.x < W) {
                hm[threadIdx.x] = s_hot[threadIdx.x];
                s_hot[threadIdx.x] = 0;
            }
            if (threadIdx.x == 0) {
                atomicAdd(&f.job.st->zr[f.d][f.i], s_zr);
                atomicAdd(&f.job.st->nhot[f.d][f.i], s_nhot);
                s_zr = 0;
                s_nhot = 0;
            }
            __syncthreads();
        }
    }
    asm volatile("cp.async.wait_group 0;" ::: "memory");
}

cudaError_t launch_plane_fold(const FoldJob &one, const FoldJob *jobs, uint32_t njobs, const Geometry &G, uint32_t ps,
                              int num_sms, cudaStream_t s) {
    if (njobs == 0) return cudaSuccess;
    const bool stats = one.st != nullptr;
    if (stats && !fold_stats_fit(G)) return cudaErrorInvalidValue;
    int per_sm = 0;
    cudaError_t e = prepare_launch(reinterpret_cast<const void *>(k_plane_fold), kFoldThreads, kFoldSmem, &per_sm);
    if (e != cudaSuccess) return e;
    uint32_t TC, W;
    fold_shape(G, stats, TC, W);
    const uint64_t rw = ((uint64_t)1 << G.k) >> 5;
    const uint64_t tiles = (uint64_t)G.dirs * G.r * (rw / W) * (G.wpc / TC) * (jobs ? njobs : 1u);
    uint64_t blocks = (uint64_t)num_sms * per_sm;
    if (tiles < blocks) blocks = tiles;
    k_plane_fold<<<(unsigned)blocks, kFoldThreads, kFoldSmem, s>>>(one, jobs, jobs ? njobs : 1u, G, ps,
                                                                   stats ? 1u : 0u);
    return cudaGetLastError();
}

}  // namespace sd
