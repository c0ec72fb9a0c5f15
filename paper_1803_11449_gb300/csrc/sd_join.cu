// sd_join.cu -- the paper's own GPU restore (§4.2, Algorithms 3 and 4): a
// staged join of the hot lists through two intermediate buffers that trade
// the reading and writing roles from one stage to the next.  An alternative
// to k_restore (tuning restore = 1); both produce K = {a : DH_i(a) in HE(i)
// for all i}.
//
// For an address a with estimators c_i = DH_i(a), Eq. 3 gives
// BL(i) = c_0 xor c_i = (a >> (i-1) alpha) mod 2^k: bits [(i-1) alpha,
// (i-1) alpha + k) of a, bits at or above 32 being zero.  So
//   stage 2 (Algorithm 3), over every (c0, c1, c2) in HE(0) x HE(1) x HE(2):
//     the high k - alpha bits of BL(1) must equal the low k - alpha bits of
//     BL(2); a surviving tuple gives bits [0, alpha + k) of a, BL(1) with the
//     high alpha bits of BL(2) above it, stored with c0;
//   stage i = 3..r-1 (Algorithm 4), over every stored (partial, c0) and every
//     c_i in HE(i): BL(i) must agree with the partial address on bits
//     [(i-1) alpha, (i-2) alpha + k) and extends it to bits [0, (i-1) alpha + k);
//   after stage r-1 the partial is all of a ((r-2) alpha + k >= 32), and a is
//     kept when DH_0(a) = c0.  The paper leaves this check implicit; without
//     it a tuple whose c0 is not a's own estimator could still yield a.
// A partial address with a bit set at or above 32 cannot extend to an
// address and is dropped at the stage that sets it; the final set is the
// same as when the check waits for the last stage.
//
// Work: |HE(0)| |HE(1)| |HE(2)| tuple tests, then |stored| |HE(i)| per
// stage.  That suits windows with small hot lists (a few hundred per row);
// k_restore does |HE(0)| |HE(1)| 2^max(0, 32-2k) tests whatever HE(2..) hold.
//
// Layout: one warp per (c0, c1) pair (stage 2) or per stored entry (later
// stages), its lanes over HE(i) 32 at a time; survivors are appended with
// one atomic per warp and ballot (the paper gives every thread a fixed share
// of the tuples and inserts one at a time).
#include "sd_common.cuh"

namespace sd {

namespace {

// Append the lanes' kept values to buf[0..cap) behind *counter, one atomic
// per warp.  The counter keeps counting past cap (the host sees overflow).
template <typename T>
__device__ __forceinline__ void warp_append(bool keep, T val, unsigned long long *counter, T *buf, uint64_t cap) {
    const uint32_t mask = __ballot_sync(0xFFFFFFFFu, keep);
    if (!mask) return;
    const uint32_t lane = threadIdx.x & 31u;
    unsigned long long base = 0;
    if (lane == 0) base = atomicAdd(counter, (unsigned long long)__popc(mask));
    base = __shfl_sync(0xFFFFFFFFu, base, 0);
    if (keep) {
        const uint64_t at = base + __popc(mask & ((1u << lane) - 1u));
        if (at < cap) buf[at] = val;
    }
}

// a[i] for a run-time i by selects (indexing the kernel parameter with a
// run-time value would copy it to local memory)
__device__ __forceinline__ uint32_t pick(const uint32_t (&a)[kMaxRows], uint32_t i) {
    uint32_t v = 0;
#pragma unroll
    for (uint32_t q = 0; q < (uint32_t)kMaxRows; q++)
        if (q == i) v = a[q];
    return v;
}

__device__ __forceinline__ const uint32_t *he_row(const Geometry &G, const JoinArgs &J, uint32_t d, uint32_t i) {
    return J.he + (((uint64_t)d * G.r + i) << G.k);
}

}  // namespace

// Stage 2: HE(0) x HE(1) x HE(2) (Algorithm 3); the last stage when r = 3.
__global__ void __launch_bounds__(256) k_join_first(Geometry G, JoinArgs J) {
    const uint32_t d = blockIdx.y;
    if (!(d ? J.run[1] : J.run[0])) return;
    const uint32_t k = G.k, al = G.alpha, ov = k - al;
    const uint32_t m = (1u << ov) - 1u;
    const uint32_t A0 = d ? G.h[1].A0 : G.h[0].A0;
    const uint32_t n0 = d ? J.n[1][0] : J.n[0][0], n1 = d ? J.n[1][1] : J.n[0][1];
    const uint32_t n2 = d ? J.n[1][2] : J.n[0][2];
    const uint32_t *he0 = he_row(G, J, d, 0), *he1 = he_row(G, J, d, 1), *he2 = he_row(G, J, d, 2);
    const bool last = G.r == 3;
    const uint32_t lane = threadIdx.x & 31u;
    const uint64_t pairs = (uint64_t)n0 * n1;
    const uint64_t nwarps = ((uint64_t)gridDim.x * blockDim.x) >> 5;
    // the list this stage fills: once past its buffer the direction is
    // overloaded and the rest of the stage is skipped (a warp-uniform read)
    const volatile unsigned long long *filled = last ? &J.stats->ncand[d] : &J.stats->jcount[d][2];
    const uint64_t fill_cap = last ? J.cand_cap : J.cap;
    for (uint64_t p = ((uint64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5; p < pairs; p += nwarps) {
        if (*filled > fill_cap) break;
        const uint32_t c0 = he0[p / n1], c1 = he1[p % n1];
        const uint32_t b1 = c0 ^ c1;  // bits [0, k) of the address
        for (uint32_t j0 = 0; j0 < n2; j0 += 32) {
            const uint32_t j = j0 + lane;
            bool keep = false;
            uint32_t a = 0;
            if (j < n2) {
                const uint32_t b2 = c0 ^ he2[j];  // bits [alpha, alpha + k)
                if ((b1 >> al) == (b2 & m)) {
                    const uint32_t hi = b2 >> ov;  // bits [k, k + alpha)
                    if (k + al <= 32 || (hi >> (32 - k)) == 0) {
                        a = b1 | (hi << k);
                        keep = true;
                    }
                }
            }
            if (last) {
                keep = keep && dh0(A0, k, a) == c0;
                warp_append<uint32_t>(keep, a, &J.stats->ncand[d], J.cand + (uint64_t)d * J.cand_cap, J.cand_cap);
            } else {
                warp_append<unsigned long long>(keep, ((unsigned long long)a << 32) | c0, &J.stats->jcount[d][2],
                                                J.sub[0] + (uint64_t)d * J.cap, J.cap);
            }
        }
    }
}

// Stage i = 3..r-1 (Algorithm 4): the entries stage i-1 stored, with HE(i).
__global__ void __launch_bounds__(256) k_join_next(Geometry G, JoinArgs J, uint32_t i) {
    const uint32_t d = blockIdx.y;
    if (!(d ? J.run[1] : J.run[0])) return;
    const uint32_t k = G.k, al = G.alpha, ov = k - al;
    const uint32_t m = (1u << ov) - 1u;
    const uint32_t A0 = d ? G.h[1].A0 : G.h[0].A0;
    const uint64_t produced = J.stats->jcount[d][i - 1];
    if (produced > J.cap) return;  // the previous stage overflowed: the direction is overloaded
    const uint64_t nin = produced;
    const unsigned long long *in = (((i - 3) & 1u) ? J.sub[1] : J.sub[0]) + (uint64_t)d * J.cap;
    unsigned long long *out = (((i - 2) & 1u) ? J.sub[1] : J.sub[0]) + (uint64_t)d * J.cap;
    const uint32_t ni = d ? pick(J.n[1], i) : pick(J.n[0], i);
    const uint32_t *hei = he_row(G, J, d, i);
    const uint32_t s_ov = (i - 1) * al;     // first address bit BL(i) shares with the partial
    const uint32_t s_new = (i - 2) * al + k;  // first address bit BL(i) adds
    const bool last = i == G.r - 1;
    const uint32_t lane = threadIdx.x & 31u;
    const uint64_t nwarps = ((uint64_t)gridDim.x * blockDim.x) >> 5;
    const volatile unsigned long long *filled = last ? &J.stats->ncand[d] : &J.stats->jcount[d][i];
    const uint64_t fill_cap = last ? J.cand_cap : J.cap;
    for (uint64_t q = ((uint64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5; q < nin; q += nwarps) {
        if (*filled > fill_cap) break;
        const unsigned long long e = in[q];
        const uint32_t part = (uint32_t)(e >> 32), c0 = (uint32_t)e;
        const uint32_t shared_bits = s_ov >= 32 ? 0u : ((part >> s_ov) & m);
        for (uint32_t j0 = 0; j0 < ni; j0 += 32) {
            const uint32_t j = j0 + lane;
            bool keep = false;
            uint32_t a = part;
            if (j < ni) {
                const uint32_t b = c0 ^ hei[j];
                if ((b & m) == shared_bits) {
                    const uint32_t hi = b >> ov;  // bits [s_new, s_new + alpha)
                    if (hi == 0) {
                        keep = true;
                    } else if (s_new < 32 && (hi >> (32 - s_new)) == 0) {
                        a = part | (hi << s_new);
                        keep = true;
                    }
                }
            }
            if (last) {
                keep = keep && dh0(A0, k, a) == c0;
                warp_append<uint32_t>(keep, a, &J.stats->ncand[d], J.cand + (uint64_t)d * J.cand_cap, J.cand_cap);
            } else {
                warp_append<unsigned long long>(keep, ((unsigned long long)a << 32) | c0, &J.stats->jcount[d][i],
                                                out, J.cap);
            }
        }
    }
}

cudaError_t launch_join(const Geometry &G, const JoinArgs &J, int num_sms, cudaStream_t s) {
    int per_sm = 0;
    cudaError_t e = prepare_launch(reinterpret_cast<const void *>(k_join_first), 256, 0, &per_sm);
    if (e != cudaSuccess) return e;
    uint64_t most = 0;
    for (uint32_t d = 0; d < G.dirs; d++)
        if (J.run[d]) most = std::max<uint64_t>(most, (uint64_t)J.n[d][0] * J.n[d][1]);
    uint64_t blocks = (uint64_t)num_sms * per_sm;
    if ((most + 7) / 8 < blocks) blocks = (most + 7) / 8;  // 8 warps per block
    if (blocks == 0) blocks = 1;
    k_join_first<<<dim3((unsigned)blocks, G.dirs), 256, 0, s>>>(G, J);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    // later stages read their input size on the device: a full grid
    e = prepare_launch(reinterpret_cast<const void *>(k_join_next), 256, 0, &per_sm);
    if (e != cudaSuccess) return e;
    for (uint32_t i = 3; i < G.r; i++) {
        k_join_next<<<dim3((unsigned)(num_sms * per_sm), G.dirs), 256, 0, s>>>(G, J, i);
        if ((e = cudaGetLastError()) != cudaSuccess) return e;
    }
    return cudaSuccess;
}

}  // namespace sd
