// Host-side internals shared by the C ABI translation units (context, plans).
#pragma once
#include "gbsieve.h"
#include "sieve_internal.cuh"

#include <cstdint>
#include <map>
#include <memory>
#include <string>
#include <vector>

namespace gbs {

constexpr uint32_t kInvBlock = 32;  // granularity of the 1/p prefix table

struct PresieveTable {
    std::vector<unsigned long long> words;  // overlapping 64-bit windows
    uint32_t modulus[kMaxPresieveGroups];
    uint32_t word_off[kMaxPresieveGroups];
    uint32_t maxp[kMaxPresieveGroups];
};
void build_presieve(PresieveTable &t);
void build_big_wheel(std::vector<uint32_t> &gapw, std::vector<uint32_t> &rstate, std::vector<uint16_t> &inv);

struct ReqSpec {
    uint64_t j0, nbits, out_word;
    uint32_t idx;
};

constexpr uint64_t kPrimePad = 64;  // zero entries allocated past the last base prime

struct Plan {
    sieve_tuning tune;
    PresieveInfo ps;
    uint32_t med_lo = 0, blk_hi = 0, coop_hi = 0;
    std::vector<TileDesc> tiles;
    std::vector<SUDesc> sus;
    std::vector<GroupDesc> groups;
    std::vector<ChunkDesc> chunks;
    struct Epoch {
        uint32_t tile0, ntiles;  // tiles [tile0, tile0+ntiles)
        uint32_t g0, ng;         // scatter groups [g0, g0+ng)
        uint32_t c0, nc;         // scatter chunks (one CTA each) [c0, c0+nc)
        uint32_t carry_base;     // first large prime index of the epoch's carried state
    };
    std::vector<Epoch> epochs;
    uint64_t pool_entries = 0;
    uint32_t max_epoch_tiles = 0;
    uint64_t carry_entries = 0;  // carried-state slots the plan needs
    bool single_request = false; // all tiles belong to one request (tile runs may carry)
    // host output: each epoch's tiles write into ring slot (epoch mod 2) of the output
    // buffer, whose slot enqueue_plan copies to host_dst + ep_word0[e] after the epoch
    bool host_out = false;
    uint64_t slot_words = 0;
    std::vector<uint64_t> ep_word0, ep_words;
    uint32_t *host_dst = nullptr;
    bool run_scatter = false;    // single-request scatter: one state word per large prime
    uint32_t state_base = 0;     //   for the whole interval, primes from index state_base
    bool big_wheel = false;      // large primes use the mod-15015 wheel (else mod 15)
    uint32_t lane_stride = 0;    // one-prime-per-thread primes of the widest tile
    uint64_t bits = 0;
    double exp_large_hits = 0;
    // count mode (sieve_count_segments): no table; per-segment prime and twin counts
    bool count_mode = false;
    unsigned long long *seg_primes = nullptr, *seg_twins = nullptr;  // caller's device counters
    uint64_t seg_j0 = 0, nsegs = 0;
    uint32_t seg_l = 0;
    uint8_t *d_edge = nullptr;   // per tile: first / last bit is a prime
    // device copies of the descriptors
    TileDesc *d_tiles = nullptr;
    SUDesc *d_sus = nullptr;
    GroupDesc *d_groups = nullptr;
    ChunkDesc *d_chunks = nullptr;
    // graph replay
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    uint32_t *g_out = nullptr;
    unsigned long long *g_counts = nullptr;
    uint64_t g_gen = 0;
    uint32_t runs = 0;
    ~Plan();
};

struct ProfRec {
    int kind;
    cudaEvent_t a, b;
};

// device scratch of one launch sequence in flight (the context owns one; each
// serving lane owns its own so that batches on different streams never share)
struct Scratch {
    // two bucket pools: the scatter of epoch e+1 fills one while the tile
    // kernel of epoch e drains the other
    uint32_t *d_bkt[2] = {nullptr, nullptr};
    size_t bkt_bytes[2] = {0, 0};
    uint32_t *d_bkt_cnt[2] = {nullptr, nullptr};  // entries per tile of the pool's epoch
    size_t bkt_cnt_bytes[2] = {0, 0};
    unsigned long long *d_ovf[2] = {nullptr, nullptr};  // overflow backstop lists
    uint32_t ovf_cap = 0;
    uint32_t *d_small = nullptr;  // [0] tile work counter, [2+b] overflow count of pool b
    int *d_err = nullptr;         // device error bits
    unsigned long long *d_acc = nullptr;  // [0] popcount, [1] profiled hits
    unsigned long long *d_carry = nullptr;  // next hit per large prime between groups
    size_t carry_bytes = 0;
    uint32_t *d_tcarry_h = nullptr;  // tile runs: next hit per (CTA, one-prime-per-thread prime)
    size_t tcarry_h_bytes = 0;
    uint64_t gen = 0;             // bumped when a buffer moves (captured graphs re-capture)
    uint64_t pool_entries = 0;    // capacity allowed per pool (entries)
    bool ext_pools = false;       // d_bkt[] point into memory the owner manages (server arena)
    cudaStream_t s_tile = nullptr, s_scat = nullptr;  // high / low priority
    cudaEvent_t ev_fork = nullptr, ev_join = nullptr, ev_scat[2] = {nullptr, nullptr},
                ev_tile[2] = {nullptr, nullptr};
};
sieve_status scratch_init(Scratch &s, uint64_t pool_entries, uint32_t ovf_cap);
void scratch_free(Scratch &s);
sieve_status scratch_ensure(Scratch &s, uint64_t pool_entries, uint32_t max_epoch_tiles,
                            uint64_t carry_entries = 0, uint64_t tile_carry_entries = 0);
}  // namespace gbs

struct sieve_ctx {
    int device = 0;
    int nsm = 0;
    uint64_t max_v = 0, base_limit = 0, nprimes = 0;
    uint32_t *d_primes = nullptr;
    uint64_t *d_barrett = nullptr;
    std::vector<uint32_t> h_primes;
    std::vector<double> h_inv_prefix;  // sum of 1/p over the first k*kInvBlock primes
    gbs::PresieveTable pre;
    unsigned long long *d_pat = nullptr;
    uint32_t *d_gapw = nullptr, *d_rstate = nullptr;  // mod-15015 wheel of the large primes
    uint16_t *d_winv = nullptr;
    sieve_tuning tune[SIEVE_TUNE_CLASSES];
    size_t mem_budget = 0;
    gbs::Scratch scr;
    unsigned long long *h_acc = nullptr;  // pinned
    int *h_err = nullptr;                 // pinned
    cudaStream_t cap_stream = nullptr;
    cudaStream_t copy_stream = nullptr;
    cudaEvent_t ev_stage[2] = {nullptr, nullptr};
    cudaEvent_t ev_copied[2] = {nullptr, nullptr};
    cudaEvent_t ev_last = nullptr;  // end of the last plan's device work (plans share the scratch)
    sieve_tuning batch_tune{};   // autotuned tuning for batches (tile_log2 == 0: class default)
    // staging for the host-output path
    uint32_t *d_stage = nullptr;
    size_t stage_bytes = 0;
    // plans
    std::map<std::string, std::unique_ptr<gbs::Plan>> plans;
    // profiling
    bool prof = false;
    bool prof_serial = false;    // profiling with scatter and tile launches on one stream
    std::vector<gbs::ProfRec> prof_recs;
    sieve_profile prof_acc{};
    int sticky_err = 0;
    // streaming (sieve_set_streaming): the large-prime state words of the last single
    // interval, valid for an interval that starts where it ended while no other plan on
    // the context's scratch has run since (carry_gen counts those runs)
    bool streaming = false;
    struct Continuation {
        bool valid = false;
        uint64_t next_J = 0;        // the first bit after the interval
        uint32_t p_lo = 0, p_hi = 0; // large primes whose state words hold their next hits
        bool big_wheel = false;
        uint64_t gen = 0;
        uint64_t scr_gen = 0;        // the scratch's buffers have not moved since
    } cont;
    uint64_t carry_gen = 0;
    const gbs::Plan *stream_plan = nullptr;  // the plan run_plan_n enqueues in streaming mode
    uint32_t stream_first_from = 0;          // its primes with state words (from p_lo)
};

namespace gbs {
extern thread_local char g_last_cuda_error[512];
uint64_t isqrt_u64(uint64_t x);
uint32_t prime_count_le(const sieve_ctx *c, uint64_t x);
double inv_sum(const sieve_ctx *c, uint32_t a, uint32_t b);
void host_prime_tables(sieve_ctx *c);
uint32_t tune_class(uint64_t vlast);
sieve_tuning default_tuning(uint32_t cls);
bool tuning_valid(const sieve_tuning &t);
std::unique_ptr<Plan> build_plan(sieve_ctx *c, const std::vector<ReqSpec> &reqs, sieve_tuning t,
                                 uint64_t pool_cap = 0);
sieve_status check_range(const sieve_ctx *c, uint64_t j0, uint64_t nbits, uint64_t *vlast);
sieve_status enqueue_plan(sieve_ctx *c, Scratch &scr, Plan *P, uint32_t *out, unsigned long long *counts,
                          uint32_t ncounts, cudaStream_t ls);
sieve_status run_plan(sieve_ctx *c, Plan *P, uint32_t *out, unsigned long long *counts, cudaStream_t st,
                      bool allow_graph);
sieve_status run_plan_n(sieve_ctx *c, Plan *P, uint32_t *out, unsigned long long *counts, uint32_t ncounts,
                        cudaStream_t st, bool allow_graph);
sieve_tuning tuning_for(const sieve_ctx *c, uint64_t vlast, uint64_t nbits);
std::string tune_key(const sieve_tuning &t);
Plan *cached_plan(sieve_ctx *c, const std::string &key, const std::vector<ReqSpec> &reqs, const sieve_tuning &t);
sieve_status upload_plan(sieve_ctx *c, Plan *P, cudaStream_t st);
}  // namespace gbs
