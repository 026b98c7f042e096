// Internal declarations of the GB300 sieve: descriptors, device helpers, launchers.
//
// Index space: absolute bit index J stands for the odd number 2J+1 (Sec. 1.2:
// only odd numbers are represented).  A prime p divides 2J+1 exactly when
// J = (p-1)/2 (mod p) (Lemma lem:q, Sec. 2.1), and its multiples are p apart in
// index space (Sec. 1.3, after the Definition).
#pragma once
#include <cstdint>
#include <cuda_runtime.h>

namespace gbs {

// ---------------------------------------------------------------------------
// Wheel W = {2,3,5} in index space (Sec. 3.2.1).  A multiple m = p*c (c odd) of a
// prime p >= 7 is struck only when c is coprime to 15: multiples with 3 | c or
// 5 | c are composites the pre-sieve already marked (3 and 5 are always in the
// first pattern group).  Stepping c -> c+2 walks the residues mod 15; the
// admissible ones, in walking order, form the cycle 1,7,11,13,2,4,8,14 with
// gaps (in steps of c -> c+2, i.e. of p in index space) 3,2,1,2,1,2,3,1.
// ---------------------------------------------------------------------------
constexpr int kWheelCycle[8] = {1, 7, 11, 13, 2, 4, 8, 14};
constexpr int kWheelGap[8] = {3, 2, 1, 2, 1, 2, 3, 1};

constexpr bool wheel_admissible(int r) { return (r % 3) != 0 && (r % 5) != 0; }
constexpr int wheel_pos(int r) {
    for (int i = 0; i < 8; ++i)
        if (kWheelCycle[i] == r) return i;
    return -1;
}
// steps (c -> c+2) from residue r to the first admissible residue
constexpr int wheel_skip(int r) {
    int k = 0;
    while (!wheel_admissible((r + 2 * k) % 15)) ++k;
    return k;
}
constexpr uint32_t pack_gap() {
    uint32_t x = 0;
    for (int s = 0; s < 8; ++s) x |= (uint32_t)kWheelGap[s] << (2 * s);
    return x;
}
constexpr uint32_t pack_skip() {
    uint32_t x = 0;
    for (int r = 0; r < 15; ++r) x |= (uint32_t)wheel_skip(r) << (2 * r);
    return x;
}
constexpr uint64_t pack_state_after_skip() {
    uint64_t x = 0;
    for (int r = 0; r < 15; ++r)
        x |= (uint64_t)wheel_pos((r + 2 * wheel_skip(r)) % 15) << (3 * r);
    return x;
}
constexpr int inv_mod15(int a) {
    for (int x = 1; x < 15; ++x)
        if ((a * x) % 15 == 1) return x;
    return 0;
}
constexpr uint64_t pack_inv15() {
    uint64_t x = 0;
    for (int r = 0; r < 15; ++r) x |= (uint64_t)inv_mod15(r) << (4 * r);
    return x;
}
// cumulative gaps: cum(s, j) = sum_{t<j} gap[(s+t)&7], 4 bits per j
constexpr uint32_t pack_cum(int s) {
    uint32_t x = 0;
    int c = 0;
    for (int j = 0; j < 8; ++j) {
        x |= (uint32_t)c << (4 * j);
        c += kWheelGap[(s + j) & 7];
    }
    return x;
}

constexpr uint32_t kGapPacked = pack_gap();
constexpr uint32_t kSkipPacked = pack_skip();
constexpr uint64_t kStateAfterPacked = pack_state_after_skip();
constexpr uint64_t kInv15Packed = pack_inv15();
static_assert(kGapPacked == 0x799Bu, "wheel gap packing");
static_assert(wheel_skip(0) == 1 && wheel_skip(3) == 2 && wheel_skip(10) == 2, "wheel skip");

__device__ __forceinline__ uint32_t wheel_gap(uint32_t s) { return (kGapPacked >> (2 * s)) & 3u; }

// ---------------------------------------------------------------------------
// 64-bit remainder by a 32-bit odd prime p without a hardware divide: Barrett
// reduction (P. Barrett, CRYPTO '86) with m = floor((2^64-1)/p) precomputed per
// prime.  q' = floor(x*m / 2^64) satisfies floor(x/p) - 1 <= q' <= floor(x/p),
// so r' = x - q'*p lies in [0, 2p) and one conditional subtraction finishes.
// ---------------------------------------------------------------------------
__device__ __forceinline__ uint32_t mod_barrett(uint64_t x, uint32_t p, uint64_t m)
{
    uint64_t q = __umul64hi(x, m);
    uint64_t r = x - q * (uint64_t)p;
    if (r >= p) r -= p;
    return (uint32_t)r;
}

// First struck index at or after Js (relative offset h from Js) for prime p,
// and the wheel state there.
//   * Lemma lem:q: the first J >= Js with p | 2J+1 is Js + q with
//     q = (p-1)/2 - (Js mod p)  (mod p).
//   * Sec. 1.4: striking with p starts at p^2, whose index is (p^2-1)/2.
//   * Sec. 3.2.1: then advance to the first multiple p*c with c coprime to 15.
// js15 = Js mod 15.  Returns h as 64-bit (the p^2 start can lie far ahead).
// Lemma lem:q: offset of the first J >= Js with p | 2J+1
__device__ __forceinline__ uint32_t lemma_q(uint64_t Js, uint32_t p, uint64_t m)
{
    const uint32_t r = mod_barrett(Js, p, m);
    const uint32_t half = p >> 1;
    return (r <= half) ? (half - r) : (half + (p - r));
}

// the rest of first_hit once q = lemma_q(Js, p, m) is known
__device__ __forceinline__ uint64_t first_hit_q(uint64_t Js, uint32_t js15, uint32_t p, uint32_t q,
                                                uint32_t &state)
{
    uint64_t jsq = ((uint64_t)p * p) >> 1;  // (p^2 - 1) / 2, p odd
    uint64_t h;
    uint32_t c15;
    if (Js + q < jsq) {
        h = jsq - Js;   // the number there is p*p, so c = p
        c15 = p % 15u;
    } else {
        h = q;
        // the number there is m = 2(Js+q)+1 = p*c, so c = m * p^{-1} (mod 15)
        uint32_t m15 = (2u * js15 + 2u * (q % 15u) + 1u) % 15u;
        uint32_t inv = (uint32_t)(kInv15Packed >> (4 * (p % 15u))) & 15u;
        c15 = (m15 * inv) % 15u;
    }
    uint32_t sk = (kSkipPacked >> (2 * c15)) & 3u;
    state = (uint32_t)(kStateAfterPacked >> (3 * c15)) & 7u;
    return h + (uint64_t)sk * p;
}

__device__ __forceinline__ uint64_t first_hit(uint64_t Js, uint32_t js15, uint32_t p, uint64_t m,
                                              uint32_t &state)
{
    return first_hit_q(Js, js15, p, lemma_q(Js, p, m), state);
}

// ---------------------------------------------------------------------------
// Big wheel for large primes: W = 3*5*7*11*13 = 15015 (all five are always in the
// first pre-sieve group), the same construction as the mod-15 wheel above but
// keeping only the 5760 multiples p*c with c coprime to 15015.  Walking c -> c+2,
// consecutive admissible residues are at most 11 steps apart, so the gaps are
// packed 8 to a 32-bit word (4 bits each); the cycle (5760) is a multiple of 8.
// Tables (built on the host, read through the L1):
//   gapw[i]    gaps of cycle positions 8i..8i+7
//   rstate[r]  for a residue r of c mod W: (steps to the first admissible residue
//              from r) << 16 | (cycle position of that residue)
//   inv[r]     r^{-1} mod W for r coprime to W
// ---------------------------------------------------------------------------
constexpr uint32_t kBigW = 15015, kBigCycle = 5760, kBigWords = kBigCycle / 8;
constexpr double kBigDensity = 5760.0 / 15015.0;  // struck multiples per multiple
struct BigWheel {
    const uint32_t *gapw;
    const uint32_t *rstate;
    const uint16_t *inv;
};

// As first_hit_q, with the mod-15015 wheel; jsw = Js mod 15015.
__device__ __forceinline__ uint64_t first_hit_big_q(uint64_t Js, uint32_t jsw, uint32_t p, uint32_t q,
                                                    const BigWheel &w, uint32_t &state)
{
    uint64_t jsq = ((uint64_t)p * p) >> 1;
    uint64_t h;
    uint32_t cw;
    if (Js + q < jsq) {
        h = jsq - Js;  // the number there is p*p, so c = p
        cw = p % kBigW;
    } else {
        h = q;
        // the number there is 2(Js+q)+1 = p*c, so c = (2(Js+q)+1) * p^{-1} (mod W)
        const uint32_t mw = (2u * jsw + 2u * (q % kBigW) + 1u) % kBigW;
        cw = (mw * (uint32_t)__ldg(w.inv + p % kBigW)) % kBigW;
    }
    const uint32_t e = __ldg(w.rstate + cw);
    state = e & 0xFFFFu;
    return h + (uint64_t)(e >> 16) * p;
}

__device__ __forceinline__ uint64_t first_hit_big(uint64_t Js, uint32_t jsw, uint32_t p, uint64_t m,
                                                  const BigWheel &w, uint32_t &state)
{
    return first_hit_big_q(Js, jsw, p, lemma_q(Js, p, m), w, state);
}

// ---------------------------------------------------------------------------
// Pre-sieve (Sec. 3.1): small primes are applied as periodic bit patterns.
// Group g covers the primes whose product is P_g; bit rho (0 <= rho < P_g + 64)
// of its pattern is 1 when some prime p of the group divides 2*rho+1 (rho = J
// mod P_g).  The pattern is stored as overlapping 64-bit words (word i holds
// bits 32i .. 32i+63), so the 32-bit window starting at rho is one load and one
// shift.
// ---------------------------------------------------------------------------
constexpr int kMaxPresieveGroups = 13;
struct PresieveInfo {
    uint32_t ngroups;                       // groups applied (1..13)
    uint32_t modulus[kMaxPresieveGroups];   // P_g
    uint32_t word_off[kMaxPresieveGroups];  // offset of the group's pattern (64-bit words)
    uint32_t max_prime;                     // largest prime covered by the applied groups
    uint64_t barrett[kMaxPresieveGroups];   // floor((2^64-1)/P_g)
    uint32_t inc[kMaxPresieveGroups];       // (32 * threads per CTA) mod P_g
    float inv[kMaxPresieveGroups];          // 1/P_g (quotient estimate, corrected exactly)
};

// ---------------------------------------------------------------------------
// Work descriptors.
// ---------------------------------------------------------------------------
struct TileDesc {
    uint64_t J;         // absolute index of the tile's first bit (multiple of 32)
    uint64_t out_word;  // word offset of the tile in the output buffer
    uint64_t bkt_off;   // entry offset of the tile's large-prime bucket in the pool
    uint32_t len;       // bits in the tile (multiple of 32, <= 2^tile_log2)
    uint32_t req;       // request index (for per-request counts)
    uint32_t bkt_cap;   // bucket capacity in entries (0: no large primes)
    uint32_t med_hi;    // medium primes used: base indices [med_lo, med_hi)
};
static_assert(sizeof(TileDesc) == 40, "TileDesc layout");

struct SUDesc {         // scatter unit: consecutive tiles of one request inside a group
    uint64_t J;         // absolute index of the first bit (start of a tile)
    uint32_t span;      // bits covered (<= 2^30)
    uint32_t tile_rel;  // index of its first tile relative to the group's first tile
    uint32_t plimit;    // largest prime that may strike (isqrt of the request's last number)
    uint32_t jw;        // J mod W of the plan's large-prime wheel (15 or 15015)
};
static_assert(sizeof(SUDesc) == 24, "SUDesc layout");

struct GroupDesc {      // scatter units sharing one flush domain (<= kScatterMaxTiles tiles)
    uint32_t su0, nsu;
    uint32_t tile0, ntiles;  // tiles [tile0, tile0+ntiles) of the launch's tile list
    uint32_t p_lo, p_hi;     // large primes: base indices [p_lo, p_hi)
    uint32_t carry_in;       // 1: unit su0 continues the previous group's last unit (same
                             // request, adjacent), so each prime's next hit is carried over
    uint32_t carry_out;      // 1: the next group continues this group's last unit
};

struct ChunkDesc {      // one scatter CTA: large primes [p_lo, p_hi), through all groups of the epoch
    uint32_t p_lo, p_hi;
};

constexpr uint32_t kStateInf = 0xFFFFFFFFu;

// device error bits
constexpr int kErrOverflow = 1;
constexpr int kErrTimeout = 2;

struct TileArgs {
    const TileDesc *tiles;
    uint32_t ntiles;
    uint32_t *work;                 // persistent-grid work counter (zeroed before launch)
    const uint32_t *primes;
    const uint64_t *barrett;
    uint32_t med_lo, blk_hi, coop_hi;  // medium primes start at med_lo; [med_lo, blk_hi) struck by
                                       // the whole CTA (each warp its slice), [blk_hi, coop_hi) one
                                       // warp per prime, the rest one thread per prime
    const unsigned long long *pat;
    PresieveInfo ps;
    const uint32_t *bkt;            // bucket pool
    const uint32_t *bkt_cnt;        // entries per tile (indexed like tiles)
    const unsigned long long *ovf;  // overflow list: (tile << 32) | offset
    const uint32_t *ovf_cnt;
    uint32_t ovf_cap;
    uint32_t *out;
    unsigned long long *req_counts; // may be null
    uint32_t tile_log2;
    // contiguous runs: CTA b takes tiles [b*run, (b+1)*run) in order and carries the
    // one-prime-per-thread primes' next hits from a tile to the next (tiles of one
    // request, each starting where the previous one ends); run = 0: work counter
    uint32_t run;
    uint32_t *carry_h;              // per CTA, per carried prime: wheel state << 29 | next hit offset
    uint32_t carry_stride;          // carried primes per CTA
    // count mode (out == null): per segment of 2^seg_l bits from seg_j0 on, the primes
    // (zero bits, the number 1 excluded) and twin pairs (adjacent zero bits, the lower
    // one in the segment) of each finished tile are added to seg_primes / seg_twins;
    // edge[t] gets bit 0 = "first bit is a prime", bit 1 = "last bit is a prime" for the
    // pairs that straddle two tiles (k_seg_edges adds those)
    unsigned long long *seg_primes;
    unsigned long long *seg_twins;
    uint8_t *edge;
    uint64_t seg_j0;
    uint32_t seg_l;
};

struct ScatterArgs {
    const uint32_t *primes;
    const uint64_t *barrett;
    const SUDesc *sus;
    const GroupDesc *groups;
    const ChunkDesc *chunks;        // one per CTA
    uint32_t ngroups;               // groups of the epoch
    const TileDesc *tiles;          // bucket offset and capacity of every tile
    unsigned long long *carry;      // per large prime (index - carry_base): next hit and wheel state
    uint32_t carry_base;
    // single-request scatter: per large prime (index - state_base) a state word that
    // lives through all epochs; run_first = 1 when group 0 is the interval's first
    unsigned long long *state;
    uint32_t state_base;
    uint32_t run_first;
    uint32_t run_last;              // 1 when the launch's last group is the interval's last (no state after it)
    uint32_t first_from;            // with run_first: primes (index - state_base) below this continue
                                    // from their state words (the previous interval ended where this
                                    // one starts); the others take a first hit
    BigWheel wheel;
    uint32_t *bkt;
    uint32_t *bkt_cnt;
    unsigned long long *ovf;
    uint32_t *ovf_cnt;
    uint32_t ovf_cap;
    int *err;
    uint32_t tile_log2;
};

// launchers (kernels.cu)
int tile_threads(uint32_t tile_log2);
int tile_blocks_per_sm(uint32_t tile_log2);
size_t tile_smem_bytes(uint32_t tile_log2);
cudaError_t launch_tiles(const TileArgs &a, uint32_t grid, cudaStream_t st);
// tiles of 2^21 bits across clusters of two CTAs (one interval, a.run tiles per cluster)
constexpr uint32_t kMaxTileLog2 = 21, kClusterTileLog2 = 21;
int ctile_max_clusters();
cudaError_t launch_ctiles(const TileArgs &a, uint32_t nclusters, cudaStream_t st);
constexpr uint32_t kScatterMaxTiles = 1024;  // tiles per scatter unit
// a scatter unit spans at most 2^30 bits (SUDesc.span), so a unit's entry v = (tile
// offset << tile_log2) + hit offset stays below 2^31 for every tile size
constexpr uint64_t kMaxUnitSpan = 1ull << 30;
static_assert(((uint64_t)kScatterMaxTiles << 20) <= kMaxUnitSpan, "a full scatter group of 2^20-bit tiles fits a unit");
// run: the single-request kernel (every group one unit continuing the previous one)
cudaError_t launch_scatter(const ScatterArgs &a, uint32_t nchunks, bool big_wheel, bool run, cudaStream_t st);
cudaError_t launch_bootstrap(uint32_t *primes_out, uint32_t *count_out, cudaStream_t st);
// primes_out holds cap entries; a count above cap writes only the first cap
cudaError_t launch_compact(const uint32_t *bits, uint64_t nbits, uint64_t jmax, uint32_t *block_cnt,
                           uint32_t *block_off, uint32_t *primes_out, uint64_t cap, uint32_t *total_out,
                           cudaStream_t st);
cudaError_t launch_barrett(const uint32_t *primes, uint64_t n, uint64_t *m, cudaStream_t st);
cudaError_t launch_popcount(const uint32_t *words, uint64_t nwords, unsigned long long *acc,
                            uint32_t grid, cudaStream_t st);
cudaError_t probe_smem_atomics(int nsm, double *atom_per_s);
cudaError_t probe_dsmem_atomics(uint32_t csize, int peer, double *atom_per_s, uint32_t *ctas);
cudaError_t set_kernel_attributes();
cudaError_t launch_sum_u32(const uint32_t *v, uint32_t n, unsigned long long *acc, cudaStream_t st);
// Goldbach search on a finished table (kernels.cu, k_goldbach): per window of
// 2^win_log2 even numbers, key = (largest minimal p) << 32 | (2^32 - 1 - offset of the
// first even number attaining it), and the count of even numbers with no p <= p_max
struct GoldbachWindow {
    unsigned long long key;
    unsigned long long failures;
};
cudaError_t launch_goldbach(const uint32_t *bits, uint64_t j0, uint64_t nwords, const uint32_t *primes,
                            uint32_t nprimes, uint64_t n_lo, uint64_t count, uint32_t win_log2, GoldbachWindow *out,
                            int nsm, cudaStream_t st);
// twin pairs across the boundary of tiles t and t+1 of one interval (count mode)
cudaError_t launch_seg_edges(const TileDesc *tiles, const uint8_t *edge, uint32_t ntiles, uint64_t seg_j0,
                             uint32_t seg_l, unsigned long long *seg_twins, cudaStream_t st);

}  // namespace gbs
