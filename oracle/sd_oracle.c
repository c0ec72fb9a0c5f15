/*
 * sd_oracle.c -- plain, single-threaded CPU oracle for DHSA super-point
 * detection ("Economical and efficient network super points detection based
 * on GPU", arxiv 1803.11449).
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing on the product path links, loads or
 * calls this file: only the test-suite, the smoke check and the benchmark's
 * CPU-baseline leg do.  It shares no code, header, table or constant
 * generator with the CUDA library; the two meet only in the written hash
 * specification below and in the grid layout that both expose.
 *
 * What each function follows:
 *   or_splitmix64, or_hash_constants ... the hash-constant reading (below)
 *   or_dh0, or_dh, or_h1 ............... DH_0 and H_1 (random hash functions,
 *                                        §3.1/§3.2) and Eq. 2 for DH_i
 *   or_update .......................... Algorithm 1 (Update DHLA)
 *   or_row_stats ....................... |LA(i,j)|, z_0 and ZR(i) (§3.3,
 *                                        first loop of Algorithm 2)
 *   or_zmin, or_hot_sets ............... Zmin and HE(i) (Algorithm 2)
 *   or_psi ............................. Lemma 1 with w' = mean of w(i)' (§3.3)
 *   or_estimate ........................ Eq. 4 (from Theorem 1)
 *   or_restore_join .................... the tuple join of Algorithm 2, in the
 *                                        staged form of Algorithms 3 and 4
 *   or_restore_preimage ................ same set, by enumerating DH_0 preimages
 *   or_close_window .................... Algorithm 2 end to end + §4.2 report
 *   or_report_brute .................... K and the report by definition, sweeping
 *                                        all 2^32 keys
 *
 * Readings of points the paper leaves open (each also recorded in the
 * project's design notes):
 *   H1, DH_0: the paper asks only for "random hash functions".  DH_0(x) is the
 *     multiply-shift family (Dietzfelbinger et al. 1997): (A0*x mod 2^32) >>
 *     (32-k), A0 odd.  H1(y) is multiply-add-shift: (A1*y + B1 mod 2^64) >>
 *     (64 - log2 g).  A0, A1, B1 are the first three outputs of splitmix64
 *     (Steele, Lea, Flood 2014) seeded with seed ^ (0x9E3779B97F4A7C15 *
 *     (dir+1)); A0 = low 32 bits | 1, A1 = output | 1, B1 = output.
 *   Eq. 2 shifts of 32 or more bits give 0.
 *   Directions: dir 0 (outbound) keys on src and hashes dst; dir 1 (inbound)
 *     keys on dst and hashes src.  Each direction has its own constants.
 *   Grid layout: uint32 words, [dir][row][cell][g/32], bit b of a cell is
 *     word b>>5, bit b&31 (LSB first).
 *   Hot: z_0 < Zmin strictly, Zmin = g*exp(-theta/g) in double.
 *   Algorithm 2 typos read as: ContainIP is set to false on a mismatch; the
 *     product in §4.2 runs over rows 0..r-1; Algorithm 4 uses CL_0 xor CL_i.
 *   Restore keeps a tuple only when the restored a0 also satisfies
 *     DH_0(a0) = CL_0, so K = { a : DH_i(a) in HE(i) for every i }.
 *   Report a0 when C(a0) >= theta (Algorithm 2 skips C < theta).
 *   Overload (the paper has no bound): a restore work bound |HE(0)|*2^(32-k),
 *     the number of keys whose DH_0 is a hot estimator of row 0, above
 *     pair_cap, or |K| > cand_cap, gives no hits for that direction and a
 *     flag.  An overloaded |K| is reported as cand_cap + 1 ("more than the
 *     cap"): the enumeration stops once it has found cand_cap + 1 members,
 *     which happens exactly when |K| > cand_cap, in whatever order K is
 *     walked.  A row with ZR(i) = 0 makes psi = 1 and Eq. 4 undefined: the
 *     direction is flagged saturated and gives no hits.
 *
 * Parity pins (tests check these against the paper and mathematics, not
 * against this code): splitmix64 published output; Eq. 2/3 round trip;
 * single-key linear-counting closed form; order/duplicate/split invariance of
 * Algorithm 1; psi in closed form for constructed grids; Eq. 4 special cases;
 * the three restore routines agree; the restored set equals an exhaustive
 * sweep of the key space; planted keys with cardinality >= 2 theta are found;
 * SZ of hand-built estimators (Definition 1).  Copies of this file with one
 * planted mistake each must fail at least one pin (the mutation tests).
 * Eq. 4 is pinned by its special cases and by inverting Theorem 1's
 * expected zero count for random g, r, c and psi (the paper prints no worked
 * example).
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

typedef struct {
    uint32_t g, r, k, alpha, dirs, reserved;
    double theta;
    uint64_t seed;
    uint64_t pair_cap; /* bound on the restore work |HE(0)|*2^(32-k) */
    uint64_t cand_cap; /* bound on |K| */
} or_params;

typedef struct {
    uint32_t A0[2];
    uint64_t A1[2];
    uint64_t B1[2];
} or_hash;

#define OR_FLAG_SATURATED 1u
#define OR_FLAG_OVERLOAD_PAIRS 2u
#define OR_FLAG_OVERLOAD_CANDS 4u

/* ---------------------------------------------------------------- hashes */

/* splitmix64: Steele, Lea, Flood, "Fast splittable pseudorandom number
 * generators" (OOPSLA 2014); the state advances by the golden-ratio gamma. */
uint64_t or_splitmix64(uint64_t *state)
{
    uint64_t z;
    *state += 0x9E3779B97F4A7C15ull;
    z = *state;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

void or_hash_constants(uint64_t seed, uint32_t dir, uint32_t *A0, uint64_t *A1, uint64_t *B1)
{
    uint64_t st = seed ^ (0x9E3779B97F4A7C15ull * (uint64_t)(dir + 1u));
    *A0 = (uint32_t)or_splitmix64(&st) | 1u;
    *A1 = or_splitmix64(&st) | 1ull;
    *B1 = or_splitmix64(&st);
}

static uint32_t log2u(uint32_t v)
{
    uint32_t l = 0;
    while ((1u << l) < v) l++;
    return l;
}

static void make_hash(const or_params *p, or_hash *h)
{
    for (uint32_t d = 0; d < 2; d++) or_hash_constants(p->seed, d, &h->A0[d], &h->A1[d], &h->B1[d]);
}

/* DH_0: maps a host uniformly into [0, 2^k). */
static inline uint32_t dh0(uint32_t A0, uint32_t k, uint32_t x)
{
    return (uint32_t)(A0 * x) >> (32u - k);
}

/* Eq. 2: DH_i(a0) = ((a0 >> (i-1)*alpha) mod 2^k) xor DH_0(a0), 1 <= i <= r-1. */
static inline uint32_t dh(uint32_t A0, uint32_t k, uint32_t alpha, uint32_t i, uint32_t x)
{
    uint32_t h0 = dh0(A0, k, x);
    uint32_t s, blk;
    if (i == 0) return h0;
    s = (i - 1u) * alpha;
    blk = (s >= 32u) ? 0u : ((x >> s) & ((1u << k) - 1u));
    return blk ^ h0;
}

uint32_t or_dh0(uint32_t A0, uint32_t k, uint32_t x) { return dh0(A0, k, x); }
uint32_t or_dh(uint32_t A0, uint32_t k, uint32_t alpha, uint32_t i, uint32_t x)
{
    return dh(A0, k, alpha, i, x);
}

/* H_1: maps a peer to a bit index in [0, g). */
uint32_t or_h1(uint64_t A1, uint64_t B1, uint32_t g, uint32_t y)
{
    return (uint32_t)((A1 * (uint64_t)y + B1) >> (64u - log2u(g)));
}

/* ---------------------------------------------------------------- checks */

/* §3.3 restrictions on r, alpha, k plus the sizes the layout supports. */
int or_check_params(const or_params *p)
{
    if (p->g < 32 || p->g > 4096 || (p->g & (p->g - 1))) return -1;
    if (p->r < 3 || p->r > 8) return -1;
    if (p->k < 1 || p->k > 24) return -1;
    if (p->alpha < 1 || p->alpha > p->k) return -1;          /* alpha <= k */
    if ((p->r - 2u) * p->alpha + p->k < 32u) return -1;      /* (r-2)alpha + k >= 32 */
    if (p->dirs < 1 || p->dirs > 2) return -1;
    if (!(p->theta > 0.0)) return -1;
    return 0;
}

static uint64_t cell_words(const or_params *p) { return p->g / 32u; }
static uint64_t row_words(const or_params *p) { return ((uint64_t)1 << p->k) * cell_words(p); }

uint64_t or_grid_words(const or_params *p) { return (uint64_t)p->dirs * p->r * row_words(p); }

static uint32_t *cell_ptr(const or_params *p, uint32_t *grid, uint32_t dir, uint32_t i, uint32_t j)
{
    return grid + ((uint64_t)dir * p->r + i) * row_words(p) + (uint64_t)j * cell_words(p);
}

/* ---------------------------------------------------------------- update */

/* Algorithm 1, applied to each pair <a0, b0> and each direction. */
void or_update(const or_params *p, uint32_t *grid, const uint32_t *pairs, uint64_t n)
{
    or_hash h;
    make_hash(p, &h);
    for (uint64_t t = 0; t < n; t++) {
        uint32_t src = pairs[2 * t], dst = pairs[2 * t + 1];
        for (uint32_t dir = 0; dir < p->dirs; dir++) {
            uint32_t a0 = dir == 0 ? src : dst;
            uint32_t b0 = dir == 0 ? dst : src;
            uint32_t BITidx = or_h1(h.A1[dir], h.B1[dir], p->g, b0);
            for (uint32_t i = 0; i < p->r; i++) {
                uint32_t LEidx = dh(h.A0[dir], p->k, p->alpha, i, a0);
                uint32_t *LEp = cell_ptr(p, grid, dir, i, LEidx);
                if ((LEp[BITidx >> 5] >> (BITidx & 31u)) & 1u) continue;
                LEp[BITidx >> 5] |= 1u << (BITidx & 31u);
            }
        }
    }
}

/* ------------------------------------------------------------- row stats */

static uint32_t weight(const uint32_t *cell, uint32_t g)
{
    uint32_t w = 0;
    for (uint32_t q = 0; q < g / 32u; q++) w += (uint32_t)__builtin_popcount(cell[q]);
    return w;
}

/* z_0(i,j) = g - |LA(i,j)| for every cell; ZR(i) = sum over j of z_0(i,j). */
void or_row_stats(const or_params *p, const uint32_t *grid, uint32_t dir, uint32_t *z0, uint64_t *zr)
{
    uint32_t ncell = 1u << p->k;
    for (uint32_t i = 0; i < p->r; i++) {
        zr[i] = 0;
        for (uint32_t j = 0; j < ncell; j++) {
            uint32_t z = p->g - weight(cell_ptr(p, (uint32_t *)grid, dir, i, j), p->g);
            z0[(uint64_t)i * ncell + j] = z;
            zr[i] += z;
        }
    }
}

/* Algorithm 2: Zmin = g * e^(-theta/g). */
double or_zmin(uint32_t g, double theta)
{
    return (double)g * exp(-theta / (double)g);
}

/* HE(i) = { j : z_0(i,j) < Zmin }, ascending j.  he holds r rows of 2^k
 * entries; nhe[i] = |HE(i)|. */
void or_hot_sets(const or_params *p, const uint32_t *z0, uint32_t *he, uint32_t *nhe)
{
    uint32_t ncell = 1u << p->k;
    double Zmin = or_zmin(p->g, p->theta);
    for (uint32_t i = 0; i < p->r; i++) {
        nhe[i] = 0;
        for (uint32_t j = 0; j < ncell; j++)
            if ((double)z0[(uint64_t)i * ncell + j] < Zmin) he[(uint64_t)i * ncell + nhe[i]++] = j;
    }
}

/* Lemma 1 with w estimated per row and averaged (§3.3):
 *   w(i)' = -g 2^k ln(ZR(i) / (g 2^k)),  w' = sum_i w(i)' / r,
 *   psi = 1 - e^(-w' / (g 2^k)).
 * Returns -1.0 when some ZR(i) = 0 (the row is saturated, Eq. 4 undefined). */
double or_psi(const or_params *p, const uint64_t *zr)
{
    double G = (double)p->g * (double)((uint64_t)1 << p->k);
    double wsum = 0.0, w;
    for (uint32_t i = 0; i < p->r; i++) {
        double wi;
        if (zr[i] == 0) return -1.0;
        wi = -G * log((double)zr[i] / G);
        wsum += wi;
    }
    w = wsum / (double)p->r;
    return 1.0 - exp(-w / G);
}

/* Eq. 4: C(a0) = -g ln( SZ(a0) / (g - g psi^r) ). */
double or_estimate(uint32_t g, uint32_t r, double psi, uint32_t sz)
{
    double gd = (double)g;
    return -gd * log((double)sz / (gd - gd * pow(psi, (double)r)));
}

/* SZ(a0): zero bits of ULE(a0), the bitwise AND of a0's r estimators (§3.2,
 * Definition 1). */
uint32_t or_sz(const or_params *p, const uint32_t *grid, uint32_t dir, uint32_t a0)
{
    or_hash h;
    uint32_t ones = 0;
    make_hash(p, &h);
    for (uint32_t q = 0; q < p->g / 32u; q++) {
        uint32_t ule = 0xFFFFFFFFu;
        for (uint32_t i = 0; i < p->r; i++) {
            uint32_t j = dh(h.A0[dir], p->k, p->alpha, i, a0);
            ule &= cell_ptr(p, (uint32_t *)grid, dir, i, j)[q];
        }
        ones += (uint32_t)__builtin_popcount(ule);
    }
    return p->g - ones;
}

/* --------------------------------------------------------------- restore */

static int cmp_u32(const void *a, const void *b)
{
    uint32_t x = *(const uint32_t *)a, y = *(const uint32_t *)b;
    return x < y ? -1 : (x > y);
}

/* hot[i] bitmap from the HE lists, for O(1) membership tests. */
static uint8_t *hot_bitmap(const or_params *p, const uint32_t *he, const uint32_t *nhe)
{
    uint32_t ncell = 1u << p->k;
    uint8_t *hot = (uint8_t *)calloc((size_t)p->r * ncell, 1);
    if (!hot) return NULL;
    for (uint32_t i = 0; i < p->r; i++)
        for (uint32_t q = 0; q < nhe[i]; q++) hot[(uint64_t)i * ncell + he[(uint64_t)i * ncell + q]] = 1;
    return hot;
}

static void emit(uint32_t *out, uint64_t cap, uint64_t *count, uint32_t a)
{
    if (*count < cap) out[*count] = a;
    (*count)++;
}

/* Algorithm 2's tuple join, in the staged form of Algorithms 3 and 4: the
 * partial address of every tuple that survives the overlap tests of rows
 * 0..i is extended by the alpha new bits of BL(i+1).  Returns |K|, writes the
 * first min(|K|, cap) members of K, ascending. */
uint64_t or_restore_join(const or_params *p, uint32_t dir, const uint32_t *he, const uint32_t *nhe,
                         uint32_t *out, uint64_t cap)
{
    uint32_t ncell = 1u << p->k, k = p->k, al = p->alpha;
    uint32_t ov = k - al;                      /* overlap k - alpha */
    uint32_t ovmask = (ov == 32u) ? 0xFFFFFFFFu : ((1u << ov) - 1u);
    const uint32_t *HE0 = he, *HE1 = he + ncell, *HE2 = he + 2 * (uint64_t)ncell;
    or_hash h;
    uint64_t nsub = 0, capsub = 1024, count = 0;
    uint32_t *sub = (uint32_t *)malloc(capsub * sizeof(uint32_t)); /* partial address */
    uint32_t *scl = (uint32_t *)malloc(capsub * sizeof(uint32_t)); /* its CL_0 */
    make_hash(p, &h);
    if (!sub || !scl) { free(sub); free(scl); return UINT64_MAX; }

    /* Algorithm 3: tuples <CL_0, CL_1, CL_2>. */
    for (uint32_t a = 0; a < nhe[0]; a++)
        for (uint32_t b = 0; b < nhe[1]; b++)
            for (uint32_t c = 0; c < nhe[2]; c++) {
                uint32_t blk1 = HE0[a] ^ HE1[b];           /* BL(1), Eq. 3 */
                uint32_t blk2 = HE0[a] ^ HE2[c];           /* BL(2), Eq. 3 */
                uint32_t hi, add;
                if ((blk1 >> al) != (blk2 & ovmask)) continue; /* left k-alpha of BL(1) vs right k-alpha of BL(2) */
                add = blk2 >> ov;                           /* the left alpha bits of BL(2) */
                /* they sit at bit k of a0; bits at 32 and above must be zero */
                if (k >= 32u) { if (add) continue; hi = 0; }
                else { if (k + al > 32u && (add >> (32u - k))) continue; hi = add << k; }
                if (nsub == capsub) {
                    capsub *= 2;
                    sub = (uint32_t *)realloc(sub, capsub * sizeof(uint32_t));
                    scl = (uint32_t *)realloc(scl, capsub * sizeof(uint32_t));
                    if (!sub || !scl) return UINT64_MAX;
                }
                sub[nsub] = blk1 | hi;
                scl[nsub] = HE0[a];
                nsub++;
            }

    /* Algorithm 4: stages i = 3..r-1 extend each partial address by BL(i). */
    for (uint32_t i = 3; i < p->r; i++) {
        const uint32_t *HEi = he + (uint64_t)i * ncell;
        uint32_t pos = (i - 2u) * al + k;      /* where the alpha new bits go */
        uint32_t top = (i - 1u) * al;           /* start of BL(i-1)'s left k-alpha bits */
        uint64_t nn = 0, capn = nsub > 0 ? nsub : 1;
        uint32_t *nsub_a = (uint32_t *)malloc(capn * sizeof(uint32_t));
        uint32_t *ncl_a = (uint32_t *)malloc(capn * sizeof(uint32_t));
        if (!nsub_a || !ncl_a) return UINT64_MAX;
        for (uint64_t s = 0; s < nsub; s++)
            for (uint32_t c = 0; c < nhe[i]; c++) {
                uint32_t blk = scl[s] ^ HEi[c];                          /* BL(i) */
                uint32_t left = top >= 32u ? 0u : ((sub[s] >> top) & ovmask);
                uint32_t add, hi;
                if (left != (blk & ovmask)) continue;
                add = blk >> ov;
                if (pos >= 32u) { if (add) continue; hi = 0; }
                else { if (pos + al > 32u && (add >> (32u - pos))) continue; hi = add << pos; }
                if (nn == capn) {
                    capn *= 2;
                    nsub_a = (uint32_t *)realloc(nsub_a, capn * sizeof(uint32_t));
                    ncl_a = (uint32_t *)realloc(ncl_a, capn * sizeof(uint32_t));
                    if (!nsub_a || !ncl_a) return UINT64_MAX;
                }
                nsub_a[nn] = sub[s] | hi;
                ncl_a[nn] = scl[s];
                nn++;
            }
        free(sub); free(scl);
        sub = nsub_a; scl = ncl_a; nsub = nn; capsub = capn;
    }

    /* restore a0 and keep it only when DH_0(a0) = CL_0 */
    for (uint64_t s = 0; s < nsub; s++)
        if (dh0(h.A0[dir], k, sub[s]) == scl[s]) emit(out, cap, &count, sub[s]);
    free(sub); free(scl);
    if (count <= cap) qsort(out, count, sizeof(uint32_t), cmp_u32);
    return count;
}

/* Multiplicative inverse of an odd A mod 2^32 by Newton's iteration
 * x <- x (2 - A x); A*A = 1 mod 8, and each step doubles the correct bits. */
uint32_t or_inverse_odd(uint32_t A)
{
    uint32_t x = A;
    for (int s = 0; s < 5; s++) x *= 2u - A * x;
    return x;
}

/* Same set K, by enumerating for each CL_0 in HE(0) the 2^(32-k) keys with
 * DH_0(a) = CL_0 (A0 is odd, so a -> A0*a mod 2^32 is a bijection) and keeping
 * those whose DH_i(a) is hot in every other row.  Returns |K| when it is at
 * most cap; otherwise stops at the first member past the cap and returns
 * cap + 1. */
uint64_t or_restore_preimage(const or_params *p, uint32_t dir, const uint32_t *he, const uint32_t *nhe,
                             uint32_t *out, uint64_t cap)
{
    uint32_t ncell = 1u << p->k, k = p->k;
    uint64_t count = 0, span = (uint64_t)1 << (32u - k);
    or_hash h;
    uint32_t A0inv;
    uint8_t *hot = hot_bitmap(p, he, nhe);
    if (!hot) return UINT64_MAX;
    make_hash(p, &h);
    A0inv = or_inverse_odd(h.A0[dir]);
    for (uint32_t q = 0; q < nhe[0]; q++) {
        uint32_t c = he[q];
        for (uint64_t t = 0; t < span; t++) {
            uint32_t a = A0inv * (((uint32_t)c << (32u - k)) | (uint32_t)t);
            int all = 1;
            for (uint32_t i = 1; i < p->r && all; i++)
                all = hot[(uint64_t)i * ncell + dh(h.A0[dir], k, p->alpha, i, a)];
            if (all) emit(out, cap, &count, a);
            if (count > cap) goto done;
        }
    }
done:
    free(hot);
    if (count <= cap) qsort(out, count, sizeof(uint32_t), cmp_u32);
    return count;
}

/* ----------------------------------------------------------- close window */

typedef struct {
    uint64_t zr[2][8];
    double psi[2];
    uint32_t n_hot[2][8];
    uint64_t n_cand[2];
    uint32_t flags[2];
    uint64_t n_hits;
} or_summary;

/* Algorithm 2 and the §4.2 estimation step for every direction: hot sets,
 * restore (DH_0-preimage form), SZ, Eq. 4, threshold.  Hits are written
 * ordered by (dir, ip), at most hit_cap of them; the return value is the
 * number of hits (which may exceed hit_cap).  cand_out, when not NULL, gets
 * K for each direction (dirs * cand_cap entries, ascending). */
uint64_t or_close_window(const or_params *p, const uint32_t *grid, or_summary *sum,
                         uint32_t *hit_dir, uint32_t *hit_ip, uint32_t *hit_sz, double *hit_est,
                         uint64_t hit_cap, uint32_t *cand_out)
{
    uint32_t ncell = 1u << p->k;
    uint32_t *z0 = (uint32_t *)malloc((size_t)p->r * ncell * sizeof(uint32_t));
    uint32_t *he = (uint32_t *)malloc((size_t)p->r * ncell * sizeof(uint32_t));
    uint64_t kcap = p->cand_cap;
    uint32_t *K = (uint32_t *)malloc((size_t)(kcap ? kcap : 1) * sizeof(uint32_t));
    uint64_t nh = 0;
    memset(sum, 0, sizeof(*sum));
    if (!z0 || !he || !K) { free(z0); free(he); free(K); return UINT64_MAX; }
    for (uint32_t dir = 0; dir < p->dirs; dir++) {
        double psi;
        uint64_t nk;
        or_row_stats(p, grid, dir, z0, sum->zr[dir]);
        or_hot_sets(p, z0, he, sum->n_hot[dir]);
        psi = or_psi(p, sum->zr[dir]);
        sum->psi[dir] = psi;
        if (psi < 0.0) { sum->flags[dir] |= OR_FLAG_SATURATED; continue; }
        if (((uint64_t)sum->n_hot[dir][0] << (32u - p->k)) > p->pair_cap) {
            sum->flags[dir] |= OR_FLAG_OVERLOAD_PAIRS;
            continue;
        }
        nk = or_restore_preimage(p, dir, he, sum->n_hot[dir], K, kcap);
        sum->n_cand[dir] = nk;
        if (nk > kcap) { sum->flags[dir] |= OR_FLAG_OVERLOAD_CANDS; continue; }
        if (cand_out) memcpy(cand_out + (uint64_t)dir * kcap, K, nk * sizeof(uint32_t));
        for (uint64_t q = 0; q < nk; q++) {
            uint32_t sz = or_sz(p, grid, dir, K[q]);
            double C = or_estimate(p->g, p->r, psi, sz);
            if (C < p->theta) continue;
            if (nh < hit_cap) {
                hit_dir[nh] = dir; hit_ip[nh] = K[q]; hit_sz[nh] = sz; hit_est[nh] = C;
            }
            nh++;
        }
    }
    sum->n_hits = nh;
    free(z0); free(he); free(K);
    return nh;
}

/* Definitional form of the report for one direction: every a in [0, 2^32)
 * whose r estimators are all hot and whose C(a) >= theta.  The same sweep
 * also yields K (all estimators hot) in out_k / *nk.  Exhaustive: tens of
 * seconds. */
uint64_t or_report_brute(const or_params *p, const uint32_t *grid, uint32_t dir,
                         uint32_t *out_ip, uint32_t *out_sz, uint64_t cap,
                         uint32_t *out_k, uint64_t kcap, uint64_t *nk)
{
    uint32_t ncell = 1u << p->k;
    uint32_t *z0 = (uint32_t *)malloc((size_t)p->r * ncell * sizeof(uint32_t));
    uint32_t *he = (uint32_t *)malloc((size_t)p->r * ncell * sizeof(uint32_t));
    uint32_t nhe[8];
    uint64_t zr[8], count = 0;
    double psi;
    or_hash h;
    uint8_t *hot;
    *nk = 0;
    if (!z0 || !he) { free(z0); free(he); return UINT64_MAX; }
    make_hash(p, &h);
    or_row_stats(p, grid, dir, z0, zr);
    or_hot_sets(p, z0, he, nhe);
    psi = or_psi(p, zr);
    hot = hot_bitmap(p, he, nhe);
    if (!hot || psi < 0.0) { free(z0); free(he); free(hot); return UINT64_MAX; }
    for (uint64_t a = 0; a < ((uint64_t)1 << 32); a++) {
        int all = 1;
        for (uint32_t i = 0; i < p->r && all; i++)
            all = hot[(uint64_t)i * ncell + dh(h.A0[dir], p->k, p->alpha, i, (uint32_t)a)];
        if (all) {
            uint32_t sz = or_sz(p, grid, dir, (uint32_t)a);
            if (*nk < kcap) out_k[*nk] = (uint32_t)a;
            (*nk)++;
            if (or_estimate(p->g, p->r, psi, sz) >= p->theta) {
                if (count < cap) { out_ip[count] = (uint32_t)a; out_sz[count] = sz; }
                count++;
            }
        }
    }
    free(z0); free(he); free(hot);
    return count;
}
