// C ABI of the GB300 sieve: context (resident base and scratch), planner,
// executor (direct launches or a replayed CUDA graph), and the entry points of
// include/gbsieve.h.
#include "gbsieve.h"
#include "sieve_internal.cuh"
#include "host_internal.h"

#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <map>
#include <memory>
#include <string>
#include <vector>

using namespace gbs;

namespace gbs {

// ---------------------------------------------------------------------------
// small exact integer helpers
// ---------------------------------------------------------------------------
uint64_t isqrt_u64(uint64_t x)
{
    if (x < 2) return x;
    uint64_t r = (uint64_t)std::sqrt((double)x);
    while ((unsigned __int128)r * r > x) --r;
    while ((unsigned __int128)(r + 1) * (r + 1) <= x) ++r;
    return r;
}

// ---------------------------------------------------------------------------
// pre-sieve groups (Sec. 3.1: small primes applied as bit masks; here as
// periodic patterns, several primes merged into one pattern as in the paper's
// 3*11 and 5*7 merge)
// ---------------------------------------------------------------------------
static const uint32_t kGroups[kMaxPresieveGroups][5] = {
    {3, 5, 7, 11, 13}, {17, 19, 23, 0, 0}, {29, 31, 0, 0, 0},  {37, 41, 0, 0, 0},  {43, 47, 0, 0, 0},
    {53, 59, 0, 0, 0}, {61, 67, 0, 0, 0},  {71, 73, 0, 0, 0},  {79, 83, 0, 0, 0},  {89, 97, 0, 0, 0},
    {101, 103, 0, 0, 0}, {107, 109, 0, 0, 0}, {113, 127, 0, 0, 0}};

void build_presieve(PresieveTable &t)
{
    t.words.clear();
    for (int g = 0; g < kMaxPresieveGroups; ++g) {
        uint32_t P = 1, maxp = 0;
        for (int i = 0; i < 5 && kGroups[g][i]; ++i) {
            P *= kGroups[g][i];
            maxp = kGroups[g][i];
        }
        t.modulus[g] = P;
        t.maxp[g] = maxp;
        t.word_off[g] = (uint32_t)t.words.size();
        // 32-bit words covering bits 0 .. P+63, then overlapping 64-bit windows
        const uint32_t nw = (P + 64 + 31) / 32 + 1;
        std::vector<uint32_t> w(nw, 0);
        for (uint32_t rho = 0; rho < 32 * nw; ++rho) {
            const uint32_t r = rho % P;  // the pattern repeats with period P
            bool hit = false;
            for (int i = 0; i < 5 && kGroups[g][i]; ++i)
                if ((2 * (uint64_t)r + 1) % kGroups[g][i] == 0) hit = true;
            if (hit) w[rho / 32] |= 1u << (rho % 32);
        }
        for (uint32_t i = 0; i + 1 < nw; ++i) t.words.push_back((unsigned long long)w[i] | ((unsigned long long)w[i + 1] << 32));
    }
}

// Tables of the mod-15015 wheel for large primes: the admissible residues of c
// (odd multiplier, p*c struck only when gcd(c, 15015) = 1) in the order in which
// stepping c -> c+2 visits them, starting from c = 1.
void build_big_wheel(std::vector<uint32_t> &gapw, std::vector<uint32_t> &rstate, std::vector<uint16_t> &inv)
{
    const uint32_t W = kBigW;
    auto coprime = [](uint32_t r) { return r % 3 && r % 5 && r % 7 && r % 11 && r % 13; };
    std::vector<int> pos(W, -1);
    std::vector<uint32_t> gap;
    uint32_t r = 1;
    do {
        pos[r] = (int)gap.size();
        uint32_t k = 1;
        while (!coprime((r + 2 * k) % W)) ++k;
        gap.push_back(k);
        r = (r + 2 * k) % W;
    } while (r != 1);
    gapw.assign(gap.size() / 8, 0);
    for (size_t i = 0; i < gap.size(); ++i) gapw[i / 8] |= gap[i] << (4 * (i % 8));
    rstate.assign(W, 0);
    for (uint32_t x = 0; x < W; ++x) {
        uint32_t k = 0;
        while (!coprime((x + 2 * k) % W)) ++k;
        rstate[x] = (k << 16) | (uint32_t)pos[(x + 2 * k) % W];
    }
    inv.assign(W, 0);
    for (uint32_t x = 1; x < W; ++x) {
        if (!coprime(x)) continue;
        // extended Euclid: t*x = 1 (mod W)
        int64_t a = x, b = W, t0 = 1, t1 = 0;
        while (b) {
            const int64_t q = a / b, ta = a - q * b, tt = t0 - q * t1;
            a = b;
            b = ta;
            t0 = t1;
            t1 = tt;
        }
        inv[x] = (uint16_t)((t0 % (int64_t)W + W) % W);
    }
}

}  // namespace gbs

// ---------------------------------------------------------------------------
// context
// ---------------------------------------------------------------------------
const char *sieve_last_cuda_error(void) { return gbs::g_last_cuda_error; }

const char *sieve_strerror(sieve_status s)
{
    switch (s) {
    case SIEVE_OK: return "ok";
    case SIEVE_EINVAL: return "invalid argument";
    case SIEVE_ERANGE: return "numbers out of range for the context";
    case SIEVE_ENOMEM: return "out of memory";
    case SIEVE_ECUDA: return "CUDA runtime error";
    case SIEVE_ETIMEOUT: return "timed out";
    case SIEVE_EBUSY: return "busy";
    case SIEVE_EOVERFLOW: return "large-prime bucket overflow";
    }
    return "unknown status";
}

// a failed CUDA runtime call: its text is kept for sieve_last_cuda_error (per thread)
#define CK(call)                                                                      \
    do {                                                                              \
        cudaError_t e_ = (call);                                                      \
        if (e_ != cudaSuccess) {                                                      \
            std::snprintf(g_last_cuda_error, sizeof g_last_cuda_error, "%s:%d %s: %s", \
                          __FILE__, __LINE__, #call, cudaGetErrorString(e_));         \
            return SIEVE_ECUDA;                                                       \
        }                                                                             \
    } while (0)

namespace gbs {
thread_local char g_last_cuda_error[512];

uint32_t prime_count_le(const sieve_ctx *c, uint64_t x)
{
    return (uint32_t)(std::upper_bound(c->h_primes.begin(), c->h_primes.end(), (uint64_t)std::min<uint64_t>(x, 0xFFFFFFFFull)) -
                      c->h_primes.begin());
}

// sum of 1/p over base indices [a, b): an upper bound from the block prefix table
double inv_sum(const sieve_ctx *c, uint32_t a, uint32_t b)
{
    if (b <= a) return 0.0;
    const uint32_t blk = kInvBlock;
    const uint32_t ba = a / blk, bb = (b + blk - 1) / blk;
    return c->h_inv_prefix[std::min<size_t>(bb, c->h_inv_prefix.size() - 1)] - c->h_inv_prefix[ba];
}

// the 1/p prefix table of the host copy of the base (chunk and bucket sizing)
void host_prime_tables(sieve_ctx *c)
{
    c->nprimes = c->h_primes.size();
    c->h_inv_prefix.assign(c->nprimes / kInvBlock + 2, 0.0);
    double acc = 0;
    for (uint64_t i = 0; i < c->nprimes; ++i) {
        if (i % kInvBlock == 0) c->h_inv_prefix[i / kInvBlock] = acc;
        acc += 1.0 / c->h_primes[i];
    }
    for (uint64_t k = (c->nprimes + kInvBlock - 1) / kInvBlock; k < c->h_inv_prefix.size(); ++k) c->h_inv_prefix[k] = acc;
}

uint32_t tune_class(uint64_t vlast)
{
    const int lg = 63 - __builtin_clzll(vlast | 1);
    return lg < 40 ? 0 : lg < 50 ? 1 : lg < 56 ? 2 : 3;
}

// defaults near what the autotuner finds on GB300 for long intervals of each class
sieve_tuning default_tuning(uint32_t cls)
{
    sieve_tuning t;
    t.tile_log2 = 20;
    t.presieve_groups = 2;
    t.coop_max = 1u << 12;
    t.medium_max = cls >= 3 ? 1u << 19 : 1u << 20;
    t.window_tiles = 1024;
    t.epoch_tiles = 4096;
    return t;  // short intervals get smaller tiles from the planner (tuning_for)
}

bool tuning_valid(const sieve_tuning &t)
{
    return t.tile_log2 >= 12 && t.tile_log2 <= kMaxTileLog2 && t.presieve_groups >= 1 &&
           t.presieve_groups <= (uint32_t)kMaxPresieveGroups && t.medium_max <= (1u << 28) &&
           t.window_tiles >= 1 && t.window_tiles <= kScatterMaxTiles &&
           ((uint64_t)t.window_tiles << t.tile_log2) <= (1ull << 30) && t.epoch_tiles >= t.window_tiles &&
           t.epoch_tiles <= 65535;
}

}  // namespace gbs

static sieve_status alloc_dev(void **p, size_t bytes)
{
    if (bytes == 0) bytes = 16;
    if (cudaMalloc(p, bytes) != cudaSuccess) {
        cudaGetLastError();
        *p = nullptr;
        return SIEVE_ENOMEM;
    }
    return SIEVE_OK;
}

// grow-only scratch buffer; *gen is bumped when the buffer moves, which makes
// captured graphs that point at the old buffer re-capture
static sieve_status ensure(void **p, size_t *have, size_t need, uint64_t *gen)
{
    if (*have >= need && *p) return SIEVE_OK;
    if (gen) ++*gen;
    if (*p) cudaDeviceSynchronize();  // in-flight work may still use it
    if (*p) cudaFree(*p);
    *p = nullptr;
    *have = 0;
    size_t n = std::max(need, (size_t)4096);
    sieve_status s = alloc_dev(p, n);
    if (s == SIEVE_OK) *have = n;
    return s;
}

namespace gbs {

sieve_status scratch_init(Scratch &s, uint64_t pool_entries, uint32_t ovf_cap)
{
    // bucket slots are addressed with 32-bit offsets inside a pool
    s.pool_entries = std::min<uint64_t>(pool_entries, (1ull << 32) - (1ull << 22));
    s.ovf_cap = ovf_cap;
    sieve_status r = alloc_dev((void **)&s.d_small, 64);
    if (!r) r = alloc_dev((void **)&s.d_err, 16);
    if (!r) r = alloc_dev((void **)&s.d_acc, 64);
    if (!r) r = alloc_dev((void **)&s.d_ovf[0], (size_t)ovf_cap * 8);
    if (!r) r = alloc_dev((void **)&s.d_ovf[1], (size_t)ovf_cap * 8);
    if (r) return r;
    CK(cudaMemset(s.d_small, 0, 64));
    CK(cudaMemset(s.d_err, 0, 16));
    CK(cudaMemset(s.d_acc, 0, 64));
    int least = 0, greatest = 0;
    CK(cudaDeviceGetStreamPriorityRange(&least, &greatest));
    CK(cudaStreamCreateWithPriority(&s.s_tile, cudaStreamNonBlocking, greatest));
    CK(cudaStreamCreateWithPriority(&s.s_scat, cudaStreamNonBlocking, least));
    CK(cudaEventCreateWithFlags(&s.ev_fork, cudaEventDisableTiming));
    CK(cudaEventCreateWithFlags(&s.ev_join, cudaEventDisableTiming));
    for (int b = 0; b < 2; ++b) {
        CK(cudaEventCreateWithFlags(&s.ev_scat[b], cudaEventDisableTiming));
        CK(cudaEventCreateWithFlags(&s.ev_tile[b], cudaEventDisableTiming));
    }
    return SIEVE_OK;
}

void scratch_free(Scratch &s)
{
    if (s.s_tile) cudaStreamSynchronize(s.s_tile);
    if (s.s_scat) cudaStreamSynchronize(s.s_scat);
    for (int b = 0; b < 2; ++b)
        for (void *p : {s.ext_pools ? nullptr : (void *)s.d_bkt[b], (void *)s.d_bkt_cnt[b], (void *)s.d_ovf[b]})
            if (p) cudaFree(p);
    if (s.d_carry) cudaFree(s.d_carry);
    if (s.d_tcarry_h) cudaFree(s.d_tcarry_h);
    for (void *p : {(void *)s.d_small, (void *)s.d_err, (void *)s.d_acc})
        if (p) cudaFree(p);
    if (s.s_tile) cudaStreamDestroy(s.s_tile);
    if (s.s_scat) cudaStreamDestroy(s.s_scat);
    for (cudaEvent_t e : {s.ev_fork, s.ev_join, s.ev_scat[0], s.ev_scat[1], s.ev_tile[0], s.ev_tile[1]})
        if (e) cudaEventDestroy(e);
    s = Scratch{};
}

sieve_status scratch_ensure(Scratch &s, uint64_t pool_entries, uint32_t max_epoch_tiles, uint64_t carry_entries,
                            uint64_t tile_carry_entries)
{
    if (pool_entries > s.pool_entries) return SIEVE_ENOMEM;
    if (tile_carry_entries) {
        sieve_status r = ensure((void **)&s.d_tcarry_h, &s.tcarry_h_bytes, (size_t)tile_carry_entries * 4, &s.gen);
        if (r) return r;
    }
    if (carry_entries) {
        sieve_status r = ensure((void **)&s.d_carry, &s.carry_bytes, (size_t)carry_entries * 8, &s.gen);
        if (r) return r;
    }
    for (int b = 0; b < 2; ++b) {
        // external pools: the owner placed them (and sized them for pool_entries)
        sieve_status r = s.ext_pools ? (s.d_bkt[b] && s.bkt_bytes[b] >= (size_t)pool_entries * 4 + 64 ? SIEVE_OK
                                                                                                  : SIEVE_ENOMEM)
                                     : ensure((void **)&s.d_bkt[b], &s.bkt_bytes[b], (size_t)pool_entries * 4 + 64,
                                              &s.gen);
        if (r) return r;
        r = ensure((void **)&s.d_bkt_cnt[b], &s.bkt_cnt_bytes[b], (size_t)max_epoch_tiles * 4 + 64, &s.gen);
        if (r) return r;
    }
    return SIEVE_OK;
}

// ---------------------------------------------------------------------------
// planner
// ---------------------------------------------------------------------------
// Every request is cut into tiles of 2^tile_log2 bits (the last one ragged).
// Requests whose largest prime exceeds medium_max also get large-prime
// buckets: their tiles are grouped into scatter groups (<= window_tiles tiles,
// runs of one request form a scatter unit) and groups into epochs whose bucket
// capacity fits the pool.  Per epoch: scatter launch, then tile launch (the
// scatter of the next epoch may overlap it, on the other bucket pool).
// Scatter chunks: each CTA takes a run of large primes through every group of
// the epoch.  Runs are cut so that every chunk of an epoch carries about the
// same estimated work: a visit per (prime, scatter unit) plus the prime's hits,
// which number span*density/p (density 8/15 or 5760/15015, the share of
// multiples the wheel keeps).  Small large primes have many hits each, so their
// chunks hold few primes.
static void make_chunks(sieve_ctx *c, Plan *P)
{
    const double kFirstHitCost = 2.0;  // one visit ~ two emitted hits
    for (Plan::Epoch &e : P->epochs) {
        e.c0 = (uint32_t)P->chunks.size();
        e.nc = 0;
        if (!e.ng) continue;
        // a chunk walks every group of the epoch: its cost is summed over groups
        std::vector<double> span(e.ng, 0.0);
        uint32_t plo = ~0u, phi = 0;
        for (uint32_t g = 0; g < e.ng; ++g) {
            const GroupDesc &G = P->groups[e.g0 + g];
            for (uint32_t k = 0; k < G.nsu; ++k) span[g] += P->sus[G.su0 + k].span;
            plo = std::min(plo, G.p_lo);
            phi = std::max(phi, G.p_hi);
        }
        auto cost = [&](uint32_t i, uint32_t j) {
            double x = 0;
            for (uint32_t g = 0; g < e.ng; ++g) {
                const GroupDesc &G = P->groups[e.g0 + g];
                const uint32_t a = std::max(i, G.p_lo), b = std::min(j, G.p_hi);
                if (a >= b) continue;
                x += kFirstHitCost * G.nsu * (double)(b - a) +
                     span[g] * (P->big_wheel ? kBigDensity : 8.0 / 15.0) * inv_sum(c, a, b);
            }
            return x;
        };
        const double target = std::max(cost(plo, phi) / (8.0 * c->nsm), 65536.0);
        uint32_t i = plo;
        while (i < phi) {
            // smallest j (step 32, at most 65536 primes) with cost(i, j) >= target
            uint32_t lo = 1, hi = std::max<uint32_t>(1, std::min<uint32_t>(2048, (phi - i + 31) / 32));
            while (lo < hi) {
                const uint32_t mid = (lo + hi) / 2;
                if (cost(i, std::min(phi, i + 32 * mid)) >= target)
                    hi = mid;
                else
                    lo = mid + 1;
            }
            const uint32_t j = std::min(phi, i + 32 * lo);
            P->chunks.push_back(ChunkDesc{i, j});
            e.nc++;
            i = j;
        }
    }
}

std::unique_ptr<Plan> build_plan(sieve_ctx *c, const std::vector<ReqSpec> &reqs, sieve_tuning t, uint64_t pool_cap_in)
{
    // cluster tiles (beyond 2^20 bits) only for one interval, whose tiles a cluster walks
    // in order; several requests take 2^20-bit tiles
    if (reqs.size() != 1 && t.tile_log2 > 20) t.tile_log2 = 20;
    const uint32_t bt = t.tile_log2;
    const uint64_t B = 1ull << bt;
    {
        // tiles, groups and epochs are addressed with 32-bit indices
        uint64_t ntiles = 0;
        for (const ReqSpec &q : reqs) ntiles += (q.nbits + B - 1) / B;
        if (ntiles >= (1ull << 31)) return nullptr;
    }
    std::unique_ptr<Plan> P(new Plan());
    P->tune = t;
    P->ps.ngroups = t.presieve_groups;
    for (int g = 0; g < kMaxPresieveGroups; ++g) {
        P->ps.modulus[g] = c->pre.modulus[g];
        P->ps.word_off[g] = c->pre.word_off[g];
        P->ps.barrett[g] = 0xFFFFFFFFFFFFFFFFull / c->pre.modulus[g];
        P->ps.inc[g] = (uint32_t)((32ull * tile_threads(t.tile_log2)) % c->pre.modulus[g]);
        P->ps.inv[g] = 1.0f / (float)c->pre.modulus[g];
    }
    P->ps.max_prime = c->pre.maxp[t.presieve_groups - 1];
    P->med_lo = prime_count_le(c, P->ps.max_prime);
    P->coop_hi = std::max(P->med_lo, prime_count_le(c, t.coop_max));
    {
        // primes whose 60-multiple warp step fits four times into the tile slice of
        // one warp are struck by the whole CTA
        // (per CTA: a cluster tile's CTAs strike these primes on their own 2^20-bit slices)
        const uint32_t nw = (uint32_t)tile_threads(t.tile_log2) / 32;
        const uint64_t cta_bits = 1ull << std::min<uint32_t>(t.tile_log2, 20);
        P->blk_hi = std::max(P->med_lo, std::min(P->coop_hi, prime_count_le(c, cta_bits / (240 * nw))));
    }
    const uint32_t large_lo = std::max(P->med_lo, prime_count_le(c, t.medium_max));
    const uint64_t pool_cap = pool_cap_in ? pool_cap_in : c->scr.pool_entries;

    struct ReqInfo {
        uint32_t med_hi, large_hi;
        double inv;
        uint32_t nsmall_large;  // large primes below the tile size (several hits per tile)
        uint32_t plimit;
    };
    std::vector<ReqInfo> info(reqs.size());
    for (size_t r = 0; r < reqs.size(); ++r) {
        const uint64_t vlast = 2 * (reqs[r].j0 + reqs[r].nbits - 1) + 1;
        const uint32_t plim = (uint32_t)isqrt_u64(vlast);
        ReqInfo &ri = info[r];
        ri.plimit = plim;
        ri.med_hi = std::max(P->med_lo, prime_count_le(c, std::min<uint64_t>(t.medium_max, plim)));
        ri.large_hi = std::max(large_lo, prime_count_le(c, plim));
        ri.inv = inv_sum(c, large_lo, ri.large_hi);
        ri.nsmall_large = ri.large_hi > large_lo
                              ? std::max(large_lo, prime_count_le(c, std::min<uint64_t>(B, plim))) - large_lo
                              : 0;
    }

    // Wheel of the large primes: the mod-15015 wheel emits 28% fewer hits than
    // the mod-15 one but its first hit costs two table reads; it pays when a
    // prime has hits in most of the units it visits (long intervals).
    {
        double hits = 0, visits = 0;
        for (size_t r = 0; r < reqs.size(); ++r) {
            if (info[r].large_hi <= large_lo) continue;
            hits += (double)reqs[r].nbits * info[r].inv;
            const double units = std::ceil((double)reqs[r].nbits / ((double)t.window_tiles * B));
            visits += units * (double)(info[r].large_hi - large_lo);
        }
        P->big_wheel = visits > 0 && hits >= 1.0 * visits;
    }
    const double density = P->big_wheel ? kBigDensity : 8.0 / 15.0;

    // tiles in request order; epochs cut at group boundaries
    Plan::Epoch ep{};
    uint64_t ep_pool = 0;
    auto close_epoch = [&]() {
        if (ep.ntiles == 0) return;
        P->epochs.push_back(ep);
        P->pool_entries = std::max(P->pool_entries, ep_pool);
        P->max_epoch_tiles = std::max(P->max_epoch_tiles, ep.ntiles);
        ep = Plan::Epoch{};
        ep.tile0 = (uint32_t)P->tiles.size();
        ep.g0 = (uint32_t)P->groups.size();
        ep_pool = 0;
    };
    ep.tile0 = 0;
    ep.g0 = 0;
    GroupDesc grp{};
    bool grp_open = false;
    auto close_group = [&]() {
        if (!grp_open) return;
        P->groups.push_back(grp);
        ep.ng++;
        grp_open = false;
    };

    // requests in order of decreasing magnitude: a scatter group then holds requests
    // that need about the same large primes, and chunks of primes above a group's
    // largest skip it (outputs do not depend on the order: every tile has its own
    // output offset and request index)
    std::vector<size_t> order(reqs.size());
    for (size_t r = 0; r < reqs.size(); ++r) order[r] = r;
    std::stable_sort(order.begin(), order.end(), [&](size_t x, size_t y) { return info[x].plimit > info[y].plimit; });
    for (size_t r : order) {
        const ReqSpec &q = reqs[r];
        const ReqInfo &ri = info[r];
        const bool large = ri.large_hi > large_lo;
        const uint64_t ntile = (q.nbits + B - 1) / B;
        P->bits += q.nbits;
        for (uint64_t k = 0; k < ntile; ++k) {
            TileDesc d{};
            d.J = q.j0 + k * B;
            d.len = (uint32_t)std::min<uint64_t>(B, q.nbits - k * B);
            d.out_word = q.out_word + (k * B) / 32;
            d.req = q.idx;
            d.med_hi = ri.med_hi;
            uint32_t cap = 0;
            if (large) {
                const double e = (double)d.len * density * ri.inv;
                cap = (uint32_t)std::ceil(1.05 * e + 8.0 * std::sqrt(e) + 64.0) + ri.nsmall_large;
                // never more than the pool holds (pools hold >= 4096 slots): hits past a
                // bucket's capacity go to the backstop list, or raise the overflow error
                cap = (uint32_t)std::min<uint64_t>((cap + 3) & ~3u, pool_cap & ~3ull);
            }
            // a new scatter group when the current one is full or this tile has no
            // large primes; a new epoch when the tile count or the pool is exhausted
            const bool new_group = !grp_open || !large || grp.ntiles >= t.window_tiles;
            const bool over = ep.ntiles >= t.epoch_tiles || ep_pool + cap > pool_cap;
            if (new_group || over) close_group();
            if (over) close_epoch();
            d.bkt_cap = cap;
            d.bkt_off = ep_pool;
            ep_pool += cap;
            const uint32_t tile_in_ep = (uint32_t)P->tiles.size() - ep.tile0;
            P->tiles.push_back(d);
            ep.ntiles++;
            if (large) {
                if (!grp_open) {
                    grp = GroupDesc{};
                    grp.su0 = (uint32_t)P->sus.size();
                    grp.tile0 = tile_in_ep;
                    grp.p_lo = large_lo;
                    grp.p_hi = large_lo;
                    grp_open = true;
                }
                // extend the group's current unit or open a new one
                const uint32_t rel = tile_in_ep - grp.tile0;
                bool extend = grp.nsu > 0;
                if (extend) {
                    SUDesc &u = P->sus.back();
                    extend = (u.J + u.span == d.J) && u.plimit == ri.plimit;
                    if (extend) u.span += d.len;
                }
                if (!extend) {
                    SUDesc u{};
                    u.J = d.J;
                    u.span = d.len;
                    u.tile_rel = rel;
                    u.plimit = ri.plimit;
                    u.jw = (uint32_t)(d.J % (P->big_wheel ? kBigW : 15u));
                    P->sus.push_back(u);
                    grp.nsu++;
                }
                grp.ntiles = rel + 1;
                grp.p_hi = std::max(grp.p_hi, ri.large_hi);
                P->exp_large_hits += (double)d.len * density * ri.inv;
            }
        }
    }
    close_group();
    close_epoch();
    for (const SUDesc &u : P->sus)
        if (u.span > kMaxUnitSpan || (uint64_t)u.tile_rel + ((u.span + B - 1) >> bt) > kScatterMaxTiles) return nullptr;
    for (const auto &e : P->epochs) P->max_epoch_tiles = std::max(P->max_epoch_tiles, e.ntiles);
    make_chunks(c, P.get());
    P->single_request = reqs.size() == 1;
    // one interval whose groups each form one unit continuing the previous group:
    // the scatter keeps one state word per large prime for the whole interval
    // (48-bit next-hit offsets: the interval stays below 2^47 bits)
    P->run_scatter = P->single_request && !P->groups.empty() && P->bits < (1ull << 47);
    for (size_t g = 0; P->run_scatter && g < P->groups.size(); ++g) {
        const GroupDesc &G = P->groups[g];
        P->run_scatter = G.nsu == 1 && G.p_lo == P->groups[0].p_lo && G.p_hi == P->groups[0].p_hi &&
                         (g == 0 || P->sus[P->groups[g - 1].su0].J + P->sus[P->groups[g - 1].su0].span ==
                                        P->sus[G.su0].J);
    }
    if (P->run_scatter) {
        P->state_base = P->groups[0].p_lo;
        // + one lane group of padding: lanes past a chunk's end load, never store
        P->carry_entries = (uint64_t)(P->groups[0].p_hi - P->groups[0].p_lo) + 32;
    }
    {
        const uint32_t lane_lo = std::max(std::max(P->med_lo, P->blk_hi), P->coop_hi);
        for (const ReqInfo &ri : info) P->lane_stride = std::max(P->lane_stride, ri.med_hi > lane_lo ? ri.med_hi - lane_lo : 0u);
    }
    // otherwise carry each prime's next hit from a group to the next when the next
    // group starts exactly where this one's last unit ends (same request) and both
    // cover the same primes (then every CTA walks both with the same primes); the
    // carried offset is 32-bit, so only inside epochs of at most 2^32 bits
    for (Plan::Epoch &e : P->epochs) {
        e.carry_base = ~0u;
        for (uint32_t g = 0; g < e.ng; ++g) e.carry_base = std::min(e.carry_base, P->groups[e.g0 + g].p_lo);
        uint64_t ebits = 0;
        for (uint32_t k = 0; k < e.ntiles; ++k) ebits += P->tiles[e.tile0 + k].len;
        if (P->run_scatter || ebits > (1ull << 32)) continue;
        for (uint32_t g = 0; g + 1 < e.ng; ++g) {
            GroupDesc &A = P->groups[e.g0 + g], &B = P->groups[e.g0 + g + 1];
            const SUDesc &ua = P->sus[A.su0 + A.nsu - 1], &ub = P->sus[B.su0];
            if (ua.J + ua.span == ub.J && ua.plimit == ub.plimit && A.p_lo == B.p_lo && A.p_hi == B.p_hi) {
                A.carry_out = 1;
                B.carry_in = 1;
                P->carry_entries = std::max<uint64_t>(P->carry_entries, A.p_hi - e.carry_base);
            }
        }
    }
    return P;
}

}  // namespace gbs

// ---------------------------------------------------------------------------
// executor
// ---------------------------------------------------------------------------
namespace gbs {

Plan::~Plan()
{
    if (exec) cudaGraphExecDestroy(exec);
    if (graph) cudaGraphDestroy(graph);
    if (d_tiles) cudaFree(d_tiles);
    if (d_sus) cudaFree(d_sus);
    if (d_groups) cudaFree(d_groups);
    if (d_chunks) cudaFree(d_chunks);
    if (d_edge) cudaFree(d_edge);
}

template <class T>
static sieve_status upload_vec(T **dst, const std::vector<T> &v, cudaStream_t st)
{
    sieve_status s = alloc_dev((void **)dst, std::max<size_t>(v.size(), 1) * sizeof(T));
    if (s) return s;
    if (!v.empty()) CK(cudaMemcpyAsync(*dst, v.data(), v.size() * sizeof(T), cudaMemcpyHostToDevice, st));
    return SIEVE_OK;
}

sieve_status upload_plan(sieve_ctx *c, Plan *P, cudaStream_t st)
{
    (void)c;
    sieve_status s = upload_vec(&P->d_tiles, P->tiles, st);
    if (!s) s = upload_vec(&P->d_sus, P->sus, st);
    if (!s) s = upload_vec(&P->d_groups, P->groups, st);
    if (!s) s = upload_vec(&P->d_chunks, P->chunks, st);
    return s;
}

static void prof_mark(sieve_ctx *c, bool on, int kind, cudaStream_t st, bool begin)
{
    if (!on) return;
    if (begin) {
        ProfRec r;
        r.kind = kind;
        cudaEventCreate(&r.a);
        cudaEventCreate(&r.b);
        cudaEventRecord(r.a, st);
        c->prof_recs.push_back(r);
    } else {
        cudaEventRecord(c->prof_recs.back().b, st);
    }
}

// The launch sequence of a plan.  The caller's stream forks into the scratch's
// tile stream (high priority) and scatter stream (low priority) and joins them
// at the end.  Epoch e uses bucket pool e%2: its scatter runs on the scatter
// stream as soon as the tile launch of epoch e-2 has drained that pool, so the
// scatter of epoch e+1 overlaps the tile launch of epoch e.
sieve_status enqueue_plan(sieve_ctx *c, Scratch &scr, Plan *P, uint32_t *out, unsigned long long *counts,
                          uint32_t ncounts, cudaStream_t ls)
{
    const uint32_t bt = P->tune.tile_log2;
    const uint32_t tgrid_max = (uint32_t)(c->nsm * tile_blocks_per_sm(bt));
    // profiling covers the context's own plans, not server lanes (their own scratch,
    // enqueued from the server's thread)
    const bool prof = c->prof && &scr == &c->scr;
    // streaming: continue from the previous interval's state words, and keep this one's
    const bool own = &scr == &c->scr;
    const bool stream_this = own && c->stream_plan == P;
    const uint32_t first_from = stream_this ? c->stream_first_from : 0u;
    if (own) {
        // this plan may overwrite the state words: no continuation survives it unless it
        // is enqueued in full as a streamed interval (recorded at the end)
        ++c->carry_gen;
        c->cont.valid = false;
    }
    cudaStream_t st = scr.s_tile, ss = prof && c->prof_serial ? scr.s_tile : scr.s_scat;
    CK(cudaEventRecord(scr.ev_fork, ls));
    CK(cudaStreamWaitEvent(st, scr.ev_fork, 0));
    CK(cudaStreamWaitEvent(ss, scr.ev_fork, 0));
    if (counts && ncounts) CK(cudaMemsetAsync(counts, 0, (size_t)ncounts * 8, st));
    if (P->count_mode) {
        CK(cudaMemsetAsync(P->seg_primes, 0, (size_t)P->nsegs * 8, st));
        if (P->seg_twins) CK(cudaMemsetAsync(P->seg_twins, 0, (size_t)P->nsegs * 8, st));
    }
    bool run_first = true;
    size_t last_scatter = 0;  // the last epoch with a scatter launch
    for (size_t ei = 0; ei < P->epochs.size(); ++ei)
        if (P->epochs[ei].ng) last_scatter = ei;
    for (size_t ei = 0; ei < P->epochs.size(); ++ei) {
        const Plan::Epoch &e = P->epochs[ei];
        const int b = (int)(ei & 1);
        if (e.ng) {
            if (ei >= 2) CK(cudaStreamWaitEvent(ss, scr.ev_tile[b], 0));
            CK(cudaMemsetAsync(scr.d_bkt_cnt[b], 0, (size_t)e.ntiles * 4, ss));
            CK(cudaMemsetAsync(scr.d_small + 2 + b, 0, 4, ss));
            ScatterArgs sa;
            sa.primes = c->d_primes;
            sa.barrett = c->d_barrett;
            sa.sus = P->d_sus;
            sa.groups = P->d_groups + e.g0;
            sa.chunks = P->d_chunks + e.c0;
            sa.ngroups = e.ng;
            sa.tiles = P->d_tiles + e.tile0;
            sa.carry = scr.d_carry;
            sa.carry_base = e.carry_base;
            sa.state = scr.d_carry;
            sa.state_base = P->state_base;
            sa.run_first = run_first ? 1u : 0u;
            sa.run_last = ei == last_scatter && !stream_this ? 1u : 0u;
            sa.first_from = first_from;
            run_first = false;
            sa.wheel.gapw = c->d_gapw;
            sa.wheel.rstate = c->d_rstate;
            sa.wheel.inv = c->d_winv;
            sa.bkt = scr.d_bkt[b];
            sa.bkt_cnt = scr.d_bkt_cnt[b];
            sa.ovf = scr.d_ovf[b];
            sa.ovf_cnt = scr.d_small + 2 + b;
            sa.ovf_cap = scr.ovf_cap;
            sa.err = scr.d_err;
            sa.tile_log2 = bt;
            prof_mark(c, prof, SIEVE_K_SCATTER, ss, true);
            CK(launch_scatter(sa, e.nc, P->big_wheel, P->run_scatter, ss));
            prof_mark(c, prof, SIEVE_K_SCATTER, ss, false);
            if (prof) CK(launch_sum_u32(scr.d_bkt_cnt[b], e.ntiles, scr.d_acc + 1, ss));
            CK(cudaEventRecord(scr.ev_scat[b], ss));
            CK(cudaStreamWaitEvent(st, scr.ev_scat[b], 0));
        }
        CK(cudaMemsetAsync(scr.d_small, 0, 4, st));
        TileArgs ta;
        ta.tiles = P->d_tiles + e.tile0;
        ta.ntiles = e.ntiles;
        ta.work = scr.d_small;
        ta.primes = c->d_primes;
        ta.barrett = c->d_barrett;
        ta.med_lo = P->med_lo;
        ta.blk_hi = P->blk_hi;
        ta.coop_hi = P->coop_hi;
        ta.pat = c->d_pat;
        ta.ps = P->ps;
        ta.bkt = scr.d_bkt[b];
        ta.bkt_cnt = scr.d_bkt_cnt[b];
        ta.ovf = scr.d_ovf[b];
        ta.ovf_cnt = scr.d_small + 2 + b;
        ta.ovf_cap = scr.ovf_cap;
        ta.out = out;
        ta.req_counts = counts;
        ta.tile_log2 = bt;
        const uint32_t tgrid = std::min<uint32_t>(e.ntiles, tgrid_max);
        ta.run = 0;
        ta.carry_h = scr.d_tcarry_h;
        ta.carry_stride = P->lane_stride;
        ta.seg_primes = P->count_mode ? P->seg_primes : nullptr;
        ta.seg_twins = P->count_mode ? P->seg_twins : nullptr;
        ta.edge = P->count_mode ? P->d_edge + e.tile0 : nullptr;
        ta.seg_j0 = P->seg_j0;
        ta.seg_l = P->seg_l;
        if (P->single_request && scr.d_tcarry_h && P->lane_stride && P->tune.medium_max <= (1u << 26)) {
            // one request: contiguous runs of tiles per CTA, carrying next hits (offsets
            // below 3 * medium_max <= 2^28 and run spans below 2^29 - 1 bits)
            const uint32_t run = (e.ntiles + tgrid - 1) / tgrid;
            if (((uint64_t)run << bt) < (1ull << 29) - 1) ta.run = run;
        }
        uint32_t nclusters = 0;
        if (bt > 20) {
            // cluster tiles: every cluster a contiguous run of tiles (both CTAs walk the
            // same ones), next hits carried inside the run
            const uint32_t maxc = (uint32_t)ctile_max_clusters();
            if (!maxc || !P->single_request || P->count_mode || (P->lane_stride && !scr.d_tcarry_h))
                return SIEVE_EINVAL;
            const uint32_t run = (e.ntiles + std::min(maxc, e.ntiles) - 1) / std::min(maxc, e.ntiles);
            if (((uint64_t)run << bt) >= (1ull << 29) - 1) return SIEVE_ERANGE;
            ta.run = run;
            nclusters = (e.ntiles + run - 1) / run;
        }
        // host output: the slot's previous copy must be done before the tiles overwrite it
        if (P->host_out && ei >= 2) CK(cudaStreamWaitEvent(st, c->ev_copied[b], 0));
        prof_mark(c, prof, SIEVE_K_TILE, st, true);
        if (bt > 20)
            CK(launch_ctiles(ta, nclusters, st));
        else
            CK(launch_tiles(ta, ta.run ? (e.ntiles + ta.run - 1) / ta.run : tgrid, st));
        prof_mark(c, prof, SIEVE_K_TILE, st, false);
        CK(cudaEventRecord(scr.ev_tile[b], st));
        if (P->host_out) {
            CK(cudaEventRecord(c->ev_stage[b], st));
            CK(cudaStreamWaitEvent(c->copy_stream, c->ev_stage[b], 0));
            prof_mark(c, prof, SIEVE_K_COPY, c->copy_stream, true);
            CK(cudaMemcpyAsync(P->host_dst + P->ep_word0[ei], out + (size_t)b * P->slot_words,
                               P->ep_words[ei] * 4, cudaMemcpyDeviceToHost, c->copy_stream));
            prof_mark(c, prof, SIEVE_K_COPY, c->copy_stream, false);
            CK(cudaEventRecord(c->ev_copied[b], c->copy_stream));
        }
    }
    // count mode: the twin pairs that straddle two tiles, once every tile is done
    if (P->count_mode && P->seg_twins)
        CK(launch_seg_edges(P->d_tiles, P->d_edge, (uint32_t)P->tiles.size(), P->seg_j0, P->seg_l, P->seg_twins, st));
    CK(cudaEventRecord(scr.ev_join, ss));
    CK(cudaStreamWaitEvent(st, scr.ev_join, 0));
    CK(cudaEventRecord(scr.ev_join, st));
    CK(cudaStreamWaitEvent(ls, scr.ev_join, 0));
    if (own) {
        if (stream_this) {
            const TileDesc &tl = P->tiles.back();
            c->cont.valid = true;
            c->cont.next_J = tl.J + tl.len;
            c->cont.p_lo = P->groups[0].p_lo;
            c->cont.p_hi = P->groups[0].p_hi;
            c->cont.big_wheel = P->big_wheel;
            c->cont.gen = c->carry_gen;
            c->cont.scr_gen = scr.gen;
        }
    }
    if (prof) {
        c->prof_acc.tiles += P->tiles.size();
        c->prof_acc.bits += P->bits;
        for (const auto &g : P->groups) c->prof_acc.prime_reads += (uint64_t)(g.p_hi - g.p_lo) * g.nsu;
        c->prof_acc.continued += first_from;
        if (P->run_scatter) {
            // the single-interval scatter writes every group's state words back but those of
            // the interval's last group, unless the interval is streamed
            size_t last = P->groups.size();
            for (size_t ei = 0; ei < P->epochs.size(); ++ei)
                if (P->epochs[ei].ng) last = P->epochs[ei].g0 + P->epochs[ei].ng - 1;
            for (size_t gi = 0; gi < P->groups.size(); ++gi)
                if (gi != last || stream_this) c->prof_acc.state_writes += P->groups[gi].p_hi - P->groups[gi].p_lo;
        }
    }
    return SIEVE_OK;
}

sieve_status run_plan_n(sieve_ctx *c, Plan *P, uint32_t *out, unsigned long long *counts, uint32_t ncounts,
                        cudaStream_t st, bool allow_graph)
{
    const uint64_t tcarry = P->single_request ? (uint64_t)c->nsm * tile_blocks_per_sm(P->tune.tile_log2) * P->lane_stride : 0;
    sieve_status s = scratch_ensure(c->scr, P->pool_entries, P->max_epoch_tiles, P->carry_entries, tcarry);
    if (s) return s;
    if (!P->d_tiles) {
        s = upload_plan(c, P, st);
        if (s) return s;
    }
    // every plan of the context shares its scratch (bucket pools, counters), so its
    // work starts after the previous plan's, whichever streams the two were issued on
    CK(cudaStreamWaitEvent(st, c->ev_last, 0));
    // streaming runs one interval after another, each plan once: no graphs
    const bool streamed = c->streaming && P->run_scatter;
    const bool graph = allow_graph && !c->prof && !streamed;
    if (graph && P->exec && P->g_out == out && P->g_counts == counts && P->g_gen == c->scr.gen) {
        ++c->carry_gen;  // the replay may overwrite the state words
        c->cont.valid = false;
        CK(cudaGraphLaunch(P->exec, st));
        CK(cudaEventRecord(c->ev_last, st));
        P->runs++;
        return SIEVE_OK;
    }
    if (graph && P->runs >= 1) {
        // second run of the same work: capture it once and replay from now on
        if (P->exec) cudaGraphExecDestroy(P->exec), P->exec = nullptr;
        if (P->graph) cudaGraphDestroy(P->graph), P->graph = nullptr;
        CK(cudaStreamBeginCapture(c->cap_stream, cudaStreamCaptureModeThreadLocal));
        sieve_status es = enqueue_plan(c, c->scr, P, out, counts, ncounts, c->cap_stream);
        cudaGraph_t g = nullptr;
        cudaError_t ce = cudaStreamEndCapture(c->cap_stream, &g);
        if (es) {
            if (g) cudaGraphDestroy(g);
            return es;
        }
        CK(ce);
        P->graph = g;
        CK(cudaGraphInstantiate(&P->exec, g, 0));
        P->g_out = out;
        P->g_counts = counts;
        P->g_gen = c->scr.gen;
        CK(cudaGraphLaunch(P->exec, st));
        CK(cudaEventRecord(c->ev_last, st));
        P->runs++;
        return SIEVE_OK;
    }
    c->stream_plan = nullptr;
    if (streamed) {
        // continue where the previous interval ended: same large primes and wheel, and its
        // state words untouched since
        const GroupDesc &G0 = P->groups[0];
        const bool ok = c->cont.valid && c->cont.gen == c->carry_gen && c->cont.scr_gen == c->scr.gen &&
                        P->tiles[0].J == c->cont.next_J && G0.p_lo == c->cont.p_lo &&
                        P->big_wheel == c->cont.big_wheel;
        c->stream_plan = P;
        c->stream_first_from = ok ? std::min(c->cont.p_hi, G0.p_hi) - G0.p_lo : 0u;
    }
    s = enqueue_plan(c, c->scr, P, out, counts, ncounts, st);
    c->stream_plan = nullptr;
    if (!s) CK(cudaEventRecord(c->ev_last, st));
    P->runs++;
    return s;
}

sieve_status run_plan(sieve_ctx *c, Plan *P, uint32_t *out, unsigned long long *counts, cudaStream_t st,
                      bool allow_graph)
{
    return run_plan_n(c, P, out, counts, 0, st, allow_graph);
}

}  // namespace gbs

// ---------------------------------------------------------------------------
// init: the base of Sec. 1.4 built on the device
// ---------------------------------------------------------------------------
static sieve_status build_base(sieve_ctx *c, cudaStream_t st)
{
    const uint64_t limit = c->base_limit;
    uint32_t *d_boot = nullptr, *d_cnt = nullptr;
    uint64_t *d_boot_m = nullptr;
    sieve_status s = alloc_dev((void **)&d_boot, 12288 * 4);
    if (!s) s = alloc_dev((void **)&d_cnt, 16);
    if (!s) s = alloc_dev((void **)&d_boot_m, 12288 * 8);
    if (s) return s;
    struct Guard {
        std::vector<void *> p;
        ~Guard() { for (void *x : p) cudaFree(x); }
    } guard;
    guard.p = {d_boot, d_cnt, d_boot_m};

    CK(launch_bootstrap(d_boot, d_cnt, st));
    uint32_t nboot = 0;
    CK(cudaMemcpyAsync(&nboot, d_cnt, 4, cudaMemcpyDeviceToHost, st));
    CK(cudaStreamSynchronize(st));
    std::vector<uint32_t> boot(nboot);
    CK(cudaMemcpy(boot.data(), d_boot, (size_t)nboot * 4, cudaMemcpyDeviceToHost));

    if (limit <= 131071) {
        const uint64_t np = std::upper_bound(boot.begin(), boot.end(), (uint32_t)limit) - boot.begin();
        c->nprimes = np;
        // + kPrimePad zero entries: the scatter's lane groups read up to 31 past a chunk
        s = alloc_dev((void **)&c->d_primes, (np + kPrimePad) * 4);
        if (s) return s;
        CK(cudaMemset(c->d_primes, 0, (np + kPrimePad) * 4));
        if (np) CK(cudaMemcpy(c->d_primes, d_boot, np * 4, cudaMemcpyDeviceToDevice));
    } else {
        // sieve indices 0..jmax (numbers 1..limit) with the bootstrap primes
        CK(launch_barrett(d_boot, nboot, d_boot_m, st));
        const uint64_t jmax = (limit - 1) / 2;
        const uint64_t nbits = (jmax + 1 + 31) / 32 * 32;
        uint32_t *d_tab = nullptr;
        s = alloc_dev((void **)&d_tab, nbits / 8 + 16);
        if (s) return s;
        guard.p.push_back(d_tab);
        const uint32_t bt = 20;
        const uint64_t B = 1ull << bt;
        std::vector<TileDesc> tiles;
        const uint32_t med_lo = (uint32_t)(std::upper_bound(boot.begin(), boot.end(), c->pre.maxp[kMaxPresieveGroups - 1]) - boot.begin());
        const uint32_t med_hi = (uint32_t)(std::upper_bound(boot.begin(), boot.end(), (uint32_t)isqrt_u64(limit)) - boot.begin());
        for (uint64_t j = 0; j < nbits; j += B) {
            TileDesc d{};
            d.J = j;
            d.len = (uint32_t)std::min<uint64_t>(B, nbits - j);
            d.out_word = j / 32;
            d.med_hi = std::max(med_lo, med_hi);
            tiles.push_back(d);
        }
        TileDesc *d_tiles = nullptr;
        s = upload_vec(&d_tiles, tiles, st);
        if (s) return s;
        guard.p.push_back(d_tiles);
        TileArgs ta{};
        ta.tiles = d_tiles;
        ta.ntiles = (uint32_t)tiles.size();
        ta.work = c->scr.d_small;
        ta.primes = d_boot;
        ta.barrett = d_boot_m;
        ta.med_lo = med_lo;
        ta.coop_hi = (uint32_t)(std::upper_bound(boot.begin(), boot.end(), 1u << 13) - boot.begin());
        ta.blk_hi = std::max(med_lo, (uint32_t)(std::upper_bound(boot.begin(), boot.end(), (uint32_t)(B / (240 * 32))) - boot.begin()));
        ta.pat = c->d_pat;
        ta.ps.ngroups = kMaxPresieveGroups;
        for (int g = 0; g < kMaxPresieveGroups; ++g) {
            ta.ps.modulus[g] = c->pre.modulus[g];
            ta.ps.word_off[g] = c->pre.word_off[g];
            ta.ps.barrett[g] = 0xFFFFFFFFFFFFFFFFull / c->pre.modulus[g];
            ta.ps.inc[g] = (uint32_t)((32ull * tile_threads(bt)) % c->pre.modulus[g]);
            ta.ps.inv[g] = 1.0f / (float)c->pre.modulus[g];
        }
        ta.ps.max_prime = c->pre.maxp[kMaxPresieveGroups - 1];
        ta.ovf_cnt = c->scr.d_small + 2;
        ta.out = d_tab;
        ta.tile_log2 = bt;
        CK(cudaMemsetAsync(c->scr.d_small, 0, 8, st));
        CK(launch_tiles(ta, std::min<uint32_t>(ta.ntiles, (uint32_t)(c->nsm * tile_blocks_per_sm(bt))), st));
        // compact the zero bits 1..jmax into the ascending prime list
        const double lx = std::log((double)limit);
        // Rosser-Schoenfeld bound on pi(x), + kPrimePad zero entries past the last prime
        const uint64_t cap = (uint64_t)(1.25506 * (double)limit / lx) + kPrimePad;
        s = alloc_dev((void **)&c->d_primes, cap * 4);
        if (s) return s;
        CK(cudaMemsetAsync(c->d_primes, 0, cap * 4, st));
        const uint64_t nwords = nbits / 32;
        const uint32_t nblocks = (uint32_t)((nwords + 4095) / 4096);
        uint32_t *d_bc = nullptr, *d_bo = nullptr;
        s = alloc_dev((void **)&d_bc, (size_t)nblocks * 4);
        if (!s) s = alloc_dev((void **)&d_bo, (size_t)nblocks * 4);
        if (s) return s;
        guard.p.push_back(d_bc);
        guard.p.push_back(d_bo);
        CK(launch_compact(d_tab, nbits, jmax, d_bc, d_bo, c->d_primes, cap, d_cnt, st));
        uint32_t np = 0;
        CK(cudaMemcpyAsync(&np, d_cnt, 4, cudaMemcpyDeviceToHost, st));
        CK(cudaStreamSynchronize(st));
        if (np + kPrimePad > cap) return SIEVE_ECUDA;
        c->nprimes = np;
    }
    s = alloc_dev((void **)&c->d_barrett, std::max<uint64_t>(c->nprimes, 1) * 8);
    if (s) return s;
    if (c->nprimes) CK(launch_barrett(c->d_primes, c->nprimes, c->d_barrett, st));
    c->h_primes.resize(c->nprimes);
    if (c->nprimes) CK(cudaMemcpyAsync(c->h_primes.data(), c->d_primes, c->nprimes * 4, cudaMemcpyDeviceToHost, st));
    CK(cudaStreamSynchronize(st));
    host_prime_tables(c);
    return SIEVE_OK;
}

sieve_status sieve_init(sieve_ctx **out, int device, uint64_t max_v, size_t mem_budget)
try {
    if (!out) return SIEVE_EINVAL;
    *out = nullptr;
    if (mem_budget && mem_budget < ((size_t)64 << 20)) return SIEVE_EINVAL;
    int ndev = 0;
    if (cudaGetDeviceCount(&ndev) != cudaSuccess || device < 0 || device >= ndev) {
        cudaGetLastError();
        return SIEVE_EINVAL;
    }
    CK(cudaSetDevice(device));
    std::unique_ptr<sieve_ctx> c(new sieve_ctx());
    c->device = device;
    CK(cudaDeviceGetAttribute(&c->nsm, cudaDevAttrMultiProcessorCount, device));
    CK(set_kernel_attributes());
    c->max_v = max_v;
    c->base_limit = std::min<uint64_t>(isqrt_u64(max_v), 0xFFFFFFFFull);
    c->mem_budget = mem_budget ? mem_budget : (size_t)16 << 30;
    build_presieve(c->pre);
    sieve_status s = alloc_dev((void **)&c->d_pat, c->pre.words.size() * 8);
    if (!s) s = scratch_init(c->scr, c->mem_budget / 8, 1u << 22);  // two pools
    if (s) {
        sieve_destroy(c.release());
        return s;
    }
    CK(cudaMemcpy(c->d_pat, c->pre.words.data(), c->pre.words.size() * 8, cudaMemcpyHostToDevice));
    {
        std::vector<uint32_t> gapw, rstate;
        std::vector<uint16_t> winv;
        build_big_wheel(gapw, rstate, winv);
        s = alloc_dev((void **)&c->d_gapw, gapw.size() * 4);
        if (!s) s = alloc_dev((void **)&c->d_rstate, rstate.size() * 4);
        if (!s) s = alloc_dev((void **)&c->d_winv, winv.size() * 2);
        if (s) {
            sieve_destroy(c.release());
            return s;
        }
        CK(cudaMemcpy(c->d_gapw, gapw.data(), gapw.size() * 4, cudaMemcpyHostToDevice));
        CK(cudaMemcpy(c->d_rstate, rstate.data(), rstate.size() * 4, cudaMemcpyHostToDevice));
        CK(cudaMemcpy(c->d_winv, winv.data(), winv.size() * 2, cudaMemcpyHostToDevice));
    }
    CK(cudaMallocHost((void **)&c->h_acc, 64));
    CK(cudaMallocHost((void **)&c->h_err, 16));
    CK(cudaStreamCreateWithFlags(&c->cap_stream, cudaStreamNonBlocking));
    CK(cudaStreamCreateWithFlags(&c->copy_stream, cudaStreamNonBlocking));
    for (int i = 0; i < 2; ++i) {
        CK(cudaEventCreateWithFlags(&c->ev_stage[i], cudaEventDisableTiming));
        CK(cudaEventCreateWithFlags(&c->ev_copied[i], cudaEventDisableTiming));
    }
    CK(cudaEventCreateWithFlags(&c->ev_last, cudaEventDisableTiming));
    for (uint32_t k = 0; k < SIEVE_TUNE_CLASSES; ++k) c->tune[k] = default_tuning(k);
    s = build_base(c.get(), c->cap_stream);
    if (s) {
        sieve_destroy(c.release());
        return s;
    }
    *out = c.release();
    return SIEVE_OK;
} catch (...) {
    return SIEVE_ENOMEM;  // host memory (or another host resource) ran out
}

void sieve_destroy(sieve_ctx *c)
{
    if (!c) return;
    cudaSetDevice(c->device);
    cudaDeviceSynchronize();
    c->plans.clear();
    for (void *p : {(void *)c->d_primes, (void *)c->d_barrett, (void *)c->d_pat, (void *)c->d_stage,
                    (void *)c->d_gapw, (void *)c->d_rstate, (void *)c->d_winv})
        if (p) cudaFree(p);
    scratch_free(c->scr);
    if (c->h_acc) cudaFreeHost(c->h_acc);
    if (c->h_err) cudaFreeHost(c->h_err);
    if (c->cap_stream) cudaStreamDestroy(c->cap_stream);
    if (c->copy_stream) cudaStreamDestroy(c->copy_stream);
    for (int i = 0; i < 2; ++i) {
        if (c->ev_stage[i]) cudaEventDestroy(c->ev_stage[i]);
        if (c->ev_copied[i]) cudaEventDestroy(c->ev_copied[i]);
    }
    if (c->ev_last) cudaEventDestroy(c->ev_last);
    for (auto &r : c->prof_recs) {
        cudaEventDestroy(r.a);
        cudaEventDestroy(r.b);
    }
    delete c;
}

// ---------------------------------------------------------------------------
// entry points
// ---------------------------------------------------------------------------
namespace gbs {

// validate an absolute range; on success *vlast = its largest number
sieve_status check_range(const sieve_ctx *c, uint64_t j0, uint64_t nbits, uint64_t *vlast)
{
    if (nbits == 0 || (j0 & 31) || (nbits & 31)) return SIEVE_EINVAL;
    const unsigned __int128 jend = (unsigned __int128)j0 + nbits;
    if (jend > ((unsigned __int128)1 << 63)) return SIEVE_ERANGE;
    const uint64_t v = (uint64_t)(2 * jend - 1);
    if (isqrt_u64(v) > c->base_limit) return SIEVE_ERANGE;
    *vlast = v;
    return SIEVE_OK;
}

// the tuning for a single interval of nbits bits: the class default, with a
// smaller tile when the interval has too few tiles to fill the GPU
sieve_tuning tuning_for(const sieve_ctx *c, uint64_t vlast, uint64_t nbits)
{
    sieve_tuning t = c->tune[tune_class(vlast)];
    while (t.tile_log2 > 14 && (nbits >> t.tile_log2) < (uint64_t)(4 * c->nsm)) {
        t.tile_log2--;
        if (t.coop_max > 64) t.coop_max >>= 1;
    }
    return t;
}

std::string tune_key(const sieve_tuning &t)
{
    char b[128];
    std::snprintf(b, sizeof b, "%u/%u/%u/%u/%u/%u", t.tile_log2, t.presieve_groups, t.coop_max, t.medium_max,
                  t.window_tiles, t.epoch_tiles);
    return b;
}

Plan *cached_plan(sieve_ctx *c, const std::string &key, const std::vector<ReqSpec> &reqs, const sieve_tuning &t)
{
    auto it = c->plans.find(key);
    if (it != c->plans.end()) return it->second.get();
    if (c->plans.size() >= 8192) {
        cudaDeviceSynchronize();
        c->plans.clear();
    }
    std::unique_ptr<Plan> P = build_plan(c, reqs, t);
    if (!P) return nullptr;
    Plan *raw = P.get();
    c->plans[key] = std::move(P);
    return raw;
}

}  // namespace gbs

sieve_status sieve_segments(sieve_ctx *c, uint32_t l, uint64_t f, uint64_t n, uint32_t *dev_bits,
                            sieve_stream stream)
try {
    if (!c || !dev_bits || l < 5 || l > 40 || n == 0 || ((uintptr_t)dev_bits & 3)) return SIEVE_EINVAL;
    if ((((unsigned __int128)f + n) << l) > ((unsigned __int128)1 << 63)) return SIEVE_ERANGE;
    const uint64_t j0 = f << l, nbits = n << l;
    uint64_t vlast;
    sieve_status s = check_range(c, j0, nbits, &vlast);
    if (s) return s;
    CK(cudaSetDevice(c->device));
    const sieve_tuning t = tuning_for(c, vlast, nbits);
    char key[160];
    std::snprintf(key, sizeof key, "S/%llu/%llu/%p/", (unsigned long long)j0, (unsigned long long)nbits,
                  (void *)dev_bits);
    std::vector<ReqSpec> reqs{{j0, nbits, 0, 0}};
    Plan *P = cached_plan(c, std::string(key) + tune_key(t), reqs, t);
    if (!P) return SIEVE_ERANGE;
    return run_plan(c, P, dev_bits, nullptr, (cudaStream_t)stream, true);
} catch (...) {
    return SIEVE_ENOMEM;  // host memory (or another host resource) ran out
}

sieve_status sieve_count_segments(sieve_ctx *c, uint32_t l, uint64_t f, uint64_t n, uint64_t *dev_primes,
                                  uint64_t *dev_twins, sieve_stream stream)
try {
    if (!c || !dev_primes || l < 12 || l > 40 || n == 0 || ((uintptr_t)dev_primes & 7) ||
        ((uintptr_t)dev_twins & 7))
        return SIEVE_EINVAL;
    if ((((unsigned __int128)f + n) << l) > ((unsigned __int128)1 << 63)) return SIEVE_ERANGE;
    const uint64_t j0 = f << l, nbits = n << l;
    uint64_t vlast;
    sieve_status s = check_range(c, j0, nbits, &vlast);
    if (s) return s;
    CK(cudaSetDevice(c->device));
    // tiles of >= 2^12 bits (tuning ranges) start 2^12-aligned relative to j0 and, since
    // 2^l >= 2^12 divides nbits, every tile is whole 4096-bit chunks of one segment
    sieve_tuning t = tuning_for(c, vlast, nbits);
    if (t.tile_log2 > 20) {
        // the count mode runs in the one-CTA tile kernel
        t.tile_log2 = 20;
        while (((uint64_t)t.window_tiles << t.tile_log2) > (1ull << 30)) t.window_tiles >>= 1;
    }
    char key[200];
    std::snprintf(key, sizeof key, "C/%llu/%llu/%u/%p/%p/", (unsigned long long)j0, (unsigned long long)nbits, l,
                  (void *)dev_primes, (void *)dev_twins);
    std::vector<ReqSpec> reqs{{j0, nbits, 0, 0}};
    Plan *P = cached_plan(c, std::string(key) + tune_key(t), reqs, t);
    if (!P) return SIEVE_ERANGE;
    if (!P->count_mode) {
        s = alloc_dev((void **)&P->d_edge, P->tiles.size());
        if (s) return s;
        P->count_mode = true;
        P->seg_primes = reinterpret_cast<unsigned long long *>(dev_primes);
        P->seg_twins = reinterpret_cast<unsigned long long *>(dev_twins);
        P->seg_j0 = j0;
        P->seg_l = l;
        P->nsegs = n;
    }
    return run_plan(c, P, nullptr, nullptr, (cudaStream_t)stream, true);
} catch (...) {
    return SIEVE_ENOMEM;  // host memory (or another host resource) ran out
}

sieve_status sieve_goldbach(sieve_ctx *c, const uint32_t *dev_bits, uint64_t j0, uint64_t nbits, uint64_t n_lo,
                            uint64_t count, uint32_t p_max, uint32_t win_log2, sieve_goldbach_window *dev_windows,
                            sieve_stream stream)
{
    static_assert(sizeof(sieve_goldbach_window) == sizeof(GoldbachWindow), "window layout");
    if (!c || !dev_bits || !dev_windows || ((uintptr_t)dev_windows & 7) || ((uintptr_t)dev_bits & 3) ||
        count == 0 || (nbits & 31) || (n_lo & 1) || n_lo < 4 || p_max < 3 || win_log2 < 5 || win_log2 > 32)
        return SIEVE_EINVAL;
    if (p_max > c->base_limit || count > (~0ull - n_lo) / 2 || j0 + nbits < j0) return SIEVE_ERANGE;
    const uint64_t n_hi = n_lo + 2 * (count - 1);
    // the largest N - 3 and, unless the table starts at 1, the smallest N - p_max lie in it
    if (n_hi / 2 - 2 >= j0 + nbits) return SIEVE_ERANGE;
    if (j0 != 0 && (n_lo / 2 < (uint64_t)(p_max + 1) / 2 + j0)) return SIEVE_ERANGE;
    CK(cudaSetDevice(c->device));
    cudaStream_t st = (cudaStream_t)stream;
    const uint64_t nwin = ((count - 1) >> win_log2) + 1;
    CK(cudaMemsetAsync(dev_windows, 0, nwin * sizeof(sieve_goldbach_window), st));
    CK(launch_goldbach(dev_bits, j0, nbits / 32, c->d_primes, prime_count_le(c, p_max), n_lo, count, win_log2,
                       reinterpret_cast<GoldbachWindow *>(dev_windows), c->nsm, st));
    return SIEVE_OK;
}

sieve_status sieve_f_from_midpoint(uint32_t l, uint64_t n, uint64_t mant, uint32_t exp10, uint64_t *f_out)
{
    if (!f_out || l < 5 || l > 40) return SIEVE_EINVAL;
    unsigned __int128 M = mant;
    for (uint32_t i = 0; i < exp10; ++i) {
        M *= 10;
        if (M >> 64) return SIEVE_ERANGE;
    }
    const unsigned __int128 q = M >> (l + 1), h = n / 2;
    *f_out = q > h ? (uint64_t)(q - h) : 0;
    return SIEVE_OK;
}

sieve_status sieve_segments_midpoint(sieve_ctx *c, uint32_t l, uint64_t mant, uint32_t exp10, uint64_t n,
                                     uint32_t *dev_bits, sieve_stream stream)
{
    uint64_t f;
    sieve_status s = sieve_f_from_midpoint(l, n, mant, exp10, &f);
    if (s) return s;
    return sieve_segments(c, l, f, n, dev_bits, stream);
}

static sieve_status take_device_error(sieve_ctx *c, cudaStream_t st)
{
    CK(cudaMemcpyAsync(c->h_err, c->scr.d_err, 4, cudaMemcpyDeviceToHost, st));
    CK(cudaStreamSynchronize(st));
    const int e = *c->h_err;
    if (e) {
        CK(cudaMemsetAsync(c->scr.d_err, 0, 4, st));
        CK(cudaStreamSynchronize(st));
        return (e & kErrTimeout) ? SIEVE_ETIMEOUT : SIEVE_EOVERFLOW;
    }
    return SIEVE_OK;
}

sieve_status sieve_sync(sieve_ctx *c, sieve_stream stream)
{
    if (!c) return SIEVE_EINVAL;
    CK(cudaSetDevice(c->device));
    CK(cudaStreamSynchronize((cudaStream_t)stream));
    CK(cudaGetLastError());
    return take_device_error(c, (cudaStream_t)stream);
}

sieve_status sieve_count(sieve_ctx *c, const uint32_t *dev_bits, uint64_t nbits, uint64_t *host_count,
                         sieve_stream stream)
{
    if (!c || !host_count || (nbits & 31) || (nbits && !dev_bits)) return SIEVE_EINVAL;
    CK(cudaSetDevice(c->device));
    cudaStream_t st = (cudaStream_t)stream;
    CK(cudaMemsetAsync(c->scr.d_acc, 0, 8, st));
    if (nbits) {
        prof_mark(c, c->prof, SIEVE_K_COUNT, st, true);
        CK(launch_popcount(dev_bits, nbits / 32, c->scr.d_acc, (uint32_t)(c->nsm * 4), st));
        prof_mark(c, c->prof, SIEVE_K_COUNT, st, false);
    }
    CK(cudaMemcpyAsync(c->h_acc, c->scr.d_acc, 8, cudaMemcpyDeviceToHost, st));
    sieve_status s = take_device_error(c, st);  // synchronises the stream
    *host_count = c->h_acc[0];
    return s;
}

sieve_status sieve_segments_host(sieve_ctx *c, uint32_t l, uint64_t f, uint64_t n, uint32_t *host_bits,
                                 sieve_stream stream)
try {
    if (!c || !host_bits || l < 5 || l > 40 || n == 0) return SIEVE_EINVAL;
    if ((((unsigned __int128)f + n) << l) > ((unsigned __int128)1 << 63)) return SIEVE_ERANGE;
    const uint64_t j0 = f << l, nbits = n << l;
    uint64_t vlast;
    sieve_status s = check_range(c, j0, nbits, &vlast);
    if (s) return s;
    CK(cudaSetDevice(c->device));
    cudaStream_t st = (cudaStream_t)stream;
    // One plan for the whole interval, epochs of at most 1024 tiles: each epoch's
    // tiles go to ring slot (epoch mod 2) in device memory and are copied to the host
    // on the copy stream while later epochs compute; a slot is reused once its copy
    // is done.  Only the last epoch's copy is not hidden behind computation.
    sieve_tuning t = tuning_for(c, vlast, nbits);
    t.epoch_tiles = std::max(t.window_tiles, std::min<uint32_t>(t.epoch_tiles, 1024));
    char key[96];
    std::snprintf(key, sizeof key, "R/%llu/%llu/", (unsigned long long)j0, (unsigned long long)nbits);
    std::vector<ReqSpec> reqs{{j0, nbits, 0, 0}};
    Plan *P = cached_plan(c, std::string(key) + tune_key(t), reqs, t);
    if (!P) return SIEVE_ERANGE;
    if (!P->host_out) {
        // first use: output offsets into the ring (descriptors are not uploaded yet)
        P->ep_word0.clear();
        P->ep_words.clear();
        uint64_t slot = 0;
        for (const Plan::Epoch &e : P->epochs) {
            uint64_t w = 0;
            for (uint32_t k = 0; k < e.ntiles; ++k) w += P->tiles[e.tile0 + k].len / 32;
            P->ep_word0.push_back(P->tiles[e.tile0].out_word);
            P->ep_words.push_back(w);
            slot = std::max<uint64_t>(slot, (w + 3) & ~3ull);  // 16-byte aligned slots
        }
        P->slot_words = slot;
        for (size_t ei = 0; ei < P->epochs.size(); ++ei) {
            const Plan::Epoch &e = P->epochs[ei];
            for (uint32_t k = 0; k < e.ntiles; ++k) {
                TileDesc &d = P->tiles[e.tile0 + k];
                d.out_word = (ei & 1) * slot + (d.out_word - P->ep_word0[ei]);
            }
        }
        P->host_out = true;
    }
    s = ensure((void **)&c->d_stage, &c->stage_bytes, 2 * P->slot_words * 4 + 64, nullptr);
    if (s) return s;
    P->host_dst = host_bits;
    s = run_plan(c, P, c->d_stage, nullptr, st, false);
    if (s) return s;
    CK(cudaStreamSynchronize(c->copy_stream));
    return sieve_sync(c, stream);
} catch (...) {
    return SIEVE_ENOMEM;  // host memory (or another host resource) ran out
}

sieve_status sieve_batch(sieve_ctx *c, const sieve_req *reqs, uint32_t count, uint32_t *dev_arena,
                         uint64_t *dev_counts, sieve_stream stream)
try {
    if (!c || (count && (!reqs || !dev_arena || !dev_counts)) || ((uintptr_t)dev_arena & 3)) return SIEVE_EINVAL;
    if (count == 0) return SIEVE_OK;
    CK(cudaSetDevice(c->device));
    std::vector<ReqSpec> rs(count);
    std::vector<uint64_t> vl(count);
    uint64_t vmax = 0, total = 0;
    // key: the request list and the output pointers
    uint64_t h = 1469598103934665603ull;
    auto mix = [&](uint64_t x) {
        for (int i = 0; i < 8; ++i) {
            h ^= (x >> (8 * i)) & 0xff;
            h *= 1099511628211ull;
        }
    };
    for (uint32_t r = 0; r < count; ++r) {
        sieve_status s = check_range(c, reqs[r].j0, reqs[r].nbits, &vl[r]);
        if (s) return s;
        rs[r] = ReqSpec{reqs[r].j0, reqs[r].nbits, reqs[r].out_word_off, r};
        vmax = std::max(vmax, vl[r]);
        total += reqs[r].nbits;
        mix(reqs[r].j0);
        mix(reqs[r].nbits);
        mix(reqs[r].out_word_off);
    }
    // largest magnitudes first: the heaviest tiles start first, and requests of
    // similar magnitude share scatter groups
    std::stable_sort(rs.begin(), rs.end(), [&](const ReqSpec &a, const ReqSpec &b) { return vl[a.idx] > vl[b.idx]; });
    sieve_tuning t = c->batch_tune.tile_log2 ? c->batch_tune : c->tune[tune_class(vmax)];
    char key[200];
    std::snprintf(key, sizeof key, "B/%u/%016llx/%p/%p/", count, (unsigned long long)h, (void *)dev_arena,
                  (void *)dev_counts);
    Plan *P = cached_plan(c, std::string(key) + tune_key(t), rs, t);
    if (!P) return SIEVE_ERANGE;
    (void)total;
    return run_plan_n(c, P, dev_arena, (unsigned long long *)dev_counts, count, (cudaStream_t)stream, true);
} catch (...) {
    return SIEVE_ENOMEM;  // host memory (or another host resource) ran out
}

sieve_status sieve_plan_describe(const uint32_t *host_primes, uint64_t nprimes, uint64_t max_v, uint32_t nsm,
                                 const sieve_req *reqs, uint32_t count, const sieve_tuning *tp,
                                 uint64_t pool_entries, sieve_plan_info *info, sieve_plan_tile *tiles,
                                 uint64_t max_tiles, sieve_plan_group *groups, uint64_t max_groups,
                                 sieve_plan_chunk *chunks, uint64_t max_chunks)
try {
    if (!info || (nprimes && !host_primes) || (count && !reqs) || nsm == 0 || nsm > 1024 ||
        pool_entries < 4096 || pool_entries > (1ull << 32) - (1ull << 22) || nprimes >= (1ull << 32) - kPrimePad)
        return SIEVE_EINVAL;
    if (tp && !tuning_valid(*tp)) return SIEVE_EINVAL;
    *info = sieve_plan_info{};
    // a host-only context: the base and the tables the planner reads, no device state
    sieve_ctx c{};
    c.nsm = (int)nsm;
    c.max_v = max_v;
    c.base_limit = std::min<uint64_t>(isqrt_u64(max_v), 0xFFFFFFFFull);
    for (uint64_t i = 0; i < nprimes; ++i)
        if (host_primes[i] < 3 || !(host_primes[i] & 1) || (i && host_primes[i] <= host_primes[i - 1]) ||
            host_primes[i] > c.base_limit)
            return SIEVE_EINVAL;
    if (count == 0) return SIEVE_OK;
    c.h_primes.assign(host_primes, host_primes + nprimes);
    host_prime_tables(&c);
    build_presieve(c.pre);
    // requests as sieve_batch takes them: checked, then largest magnitude first
    std::vector<ReqSpec> rs(count);
    std::vector<uint64_t> vl(count);
    uint64_t vmax = 0;
    for (uint32_t r = 0; r < count; ++r) {
        sieve_status s = check_range(&c, reqs[r].j0, reqs[r].nbits, &vl[r]);
        if (s) return s;
        rs[r] = ReqSpec{reqs[r].j0, reqs[r].nbits, reqs[r].out_word_off, r};
        vmax = std::max(vmax, vl[r]);
    }
    std::stable_sort(rs.begin(), rs.end(), [&](const ReqSpec &a, const ReqSpec &b) { return vl[a.idx] > vl[b.idx]; });
    for (uint32_t k = 0; k < SIEVE_TUNE_CLASSES; ++k) c.tune[k] = default_tuning(k);
    // no tuning given: what a fresh context takes (sieve_segments' for one interval)
    const sieve_tuning t = tp ? *tp : count == 1 ? tuning_for(&c, vl[0], reqs[0].nbits) : c.tune[tune_class(vmax)];
    std::unique_ptr<Plan> P = build_plan(&c, rs, t, pool_entries);
    if (!P) return SIEVE_ERANGE;

    info->ntiles = P->tiles.size();
    info->ngroups = P->groups.size();
    info->nepochs = P->epochs.size();
    info->nchunks = P->chunks.size();
    info->nunits = P->sus.size();
    info->bits = P->bits;
    info->pool_entries = P->pool_entries;
    info->carry_entries = P->carry_entries;
    info->max_epoch_tiles = P->max_epoch_tiles;
    info->big_wheel = P->big_wheel;
    info->run_scatter = P->run_scatter;
    for (const GroupDesc &G : P->groups) info->carried_groups += G.carry_in;
    info->med_lo = P->med_lo;
    info->blk_hi = P->blk_hi;
    info->coop_hi = P->coop_hi;
    info->large_lo = std::max(P->med_lo, prime_count_le(&c, t.medium_max));
    info->expected_large_hits = P->exp_large_hits;

    std::vector<uint32_t> tile_group(P->tiles.size(), 0xFFFFFFFFu), tile_epoch(P->tiles.size(), 0);
    for (uint32_t e = 0; e < P->epochs.size(); ++e) {
        const Plan::Epoch &E = P->epochs[e];
        for (uint32_t k = 0; k < E.ntiles; ++k) tile_epoch[E.tile0 + k] = e;
        for (uint32_t g = 0; g < E.ng; ++g) {
            const GroupDesc &G = P->groups[E.g0 + g];
            for (uint32_t k = 0; k < G.ntiles; ++k) tile_group[E.tile0 + G.tile0 + k] = E.g0 + g;
            if (groups && E.g0 + g < max_groups)
                groups[E.g0 + g] = sieve_plan_group{e, E.tile0 + G.tile0, G.ntiles, G.nsu, G.p_lo, G.p_hi,
                                                    G.carry_in, G.carry_out};
        }
        for (uint32_t k = 0; k < E.nc; ++k)
            if (chunks && E.c0 + k < max_chunks)
                chunks[E.c0 + k] = sieve_plan_chunk{e, P->chunks[E.c0 + k].p_lo, P->chunks[E.c0 + k].p_hi};
    }
    for (uint64_t i = 0; tiles && i < std::min<uint64_t>(max_tiles, P->tiles.size()); ++i) {
        const TileDesc &d = P->tiles[i];
        tiles[i] = sieve_plan_tile{d.J, d.out_word, d.bkt_off, d.len, d.req, tile_epoch[i], tile_group[i],
                                   d.bkt_cap, d.med_hi};
    }
    return SIEVE_OK;
} catch (...) {
    return SIEVE_ENOMEM;  // host memory (or another host resource) ran out
}

sieve_status sieve_get_tuning(sieve_ctx *c, uint32_t cls, sieve_tuning *out)
{
    if (!c || !out || cls >= SIEVE_TUNE_CLASSES) return SIEVE_EINVAL;
    *out = c->tune[cls];
    return SIEVE_OK;
}

sieve_status sieve_set_tuning(sieve_ctx *c, uint32_t cls, const sieve_tuning *in)
{
    if (!c || !in || cls >= SIEVE_TUNE_CLASSES || !tuning_valid(*in)) return SIEVE_EINVAL;
    c->tune[cls] = *in;
    c->batch_tune = sieve_tuning{};  // an explicit tuning replaces the autotuned batch one
    return SIEVE_OK;
}

sieve_status sieve_base_info(sieve_ctx *c, const uint32_t **dev_primes, uint64_t *count, uint64_t *limit)
{
    if (!c) return SIEVE_EINVAL;
    if (dev_primes) *dev_primes = c->d_primes;
    if (count) *count = c->nprimes;
    if (limit) *limit = c->base_limit;
    return SIEVE_OK;
}

sieve_status sieve_profile_enable(sieve_ctx *c, int enable)
{
    if (!c) return SIEVE_EINVAL;
    c->prof = enable != 0;
    c->prof_serial = enable == 2;
    return SIEVE_OK;
}

sieve_status sieve_profile_read(sieve_ctx *c, sieve_profile *out, sieve_stream stream)
try {
    if (!c || !out) return SIEVE_EINVAL;
    CK(cudaSetDevice(c->device));
    CK(cudaStreamSynchronize((cudaStream_t)stream));
    CK(cudaStreamSynchronize(c->copy_stream));
    for (auto &r : c->prof_recs) {
        float ms = 0;
        CK(cudaEventSynchronize(r.b));
        CK(cudaEventElapsedTime(&ms, r.a, r.b));
        if (r.kind >= 0 && r.kind < 8) {
            c->prof_acc.launches[r.kind]++;
            c->prof_acc.ms[r.kind] += ms;
        }
        cudaEventDestroy(r.a);
        cudaEventDestroy(r.b);
    }
    c->prof_recs.clear();
    CK(cudaMemcpy(c->h_acc, c->scr.d_acc, 16, cudaMemcpyDeviceToHost));
    c->prof_acc.large_hits = c->h_acc[1];
    *out = c->prof_acc;
    c->prof_acc = sieve_profile{};
    CK(cudaMemset(c->scr.d_acc + 1, 0, 8));
    return SIEVE_OK;
} catch (...) {
    return SIEVE_ENOMEM;  // host memory (or another host resource) ran out
}

sieve_status sieve_probe_smem_atomics(int device, double *atomics_per_s)
{
    if (!atomics_per_s) return SIEVE_EINVAL;
    CK(cudaSetDevice(device));
    int nsm = 0;
    CK(cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, device));
    CK(probe_smem_atomics(nsm, atomics_per_s));
    return SIEVE_OK;
}

sieve_status sieve_probe_dsmem_atomics(int device, uint32_t cluster_size, int peer, double *atomics_per_s,
                                       uint32_t *ctas)
{
    if (!atomics_per_s || !ctas || cluster_size < 2 || cluster_size > 8 || (cluster_size & (cluster_size - 1)))
        return SIEVE_EINVAL;
    CK(cudaSetDevice(device));
    CK(probe_dsmem_atomics(cluster_size, peer ? 1 : 0, atomics_per_s, ctas));
    return SIEVE_OK;
}

sieve_status sieve_set_streaming(sieve_ctx *c, int enable)
{
    if (!c) return SIEVE_EINVAL;
    c->streaming = enable != 0;
    c->cont.valid = false;
    return SIEVE_OK;
}
