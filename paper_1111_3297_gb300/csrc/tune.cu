// Autotuner: times candidate tunings of the device path on the caller's own
// workload and keeps the fastest.  The bits never depend on the tuning; only
// the time does.
#include "gbsieve.h"
#include "host_internal.h"

#include <algorithm>
#include <vector>

using namespace gbs;

namespace {

struct Timer {
    cudaEvent_t a = nullptr, b = nullptr;
    Timer() {
        cudaEventCreate(&a);
        cudaEventCreate(&b);
    }
    ~Timer() {
        cudaEventDestroy(a);
        cudaEventDestroy(b);
    }
};

// best of `reps` timed runs (after one untimed run) of the work `reqs` under
// tuning t; +inf when the tuning does not fit the memory budget
double time_tuning(sieve_ctx *c, const std::vector<ReqSpec> &reqs, const sieve_tuning &t, uint32_t *out,
                   unsigned long long *counts, uint32_t ncounts, cudaStream_t st, int reps)
{
    std::unique_ptr<Plan> P = build_plan(c, reqs, t);
    if (!P || P->pool_entries > c->scr.pool_entries) return 1e30;
    if (run_plan_n(c, P.get(), out, counts, ncounts, st, false) != SIEVE_OK) return 1e30;
    Timer tm;
    double best = 1e30;
    for (int r = 0; r < reps; ++r) {
        cudaEventRecord(tm.a, st);
        if (enqueue_plan(c, c->scr, P.get(), out, counts, ncounts, st) != SIEVE_OK) return 1e30;
        cudaEventRecord(tm.b, st);
        if (cudaEventSynchronize(tm.b) != cudaSuccess) return 1e30;
        float ms = 0;
        cudaEventElapsedTime(&ms, tm.a, tm.b);
        best = std::min(best, (double)ms);
    }
    cudaStreamSynchronize(st);  // the plan's descriptors are freed with it
    return best;
}

// coordinate descent over the tuning parameters, two passes
sieve_tuning descend(sieve_ctx *c, const std::vector<ReqSpec> &reqs, sieve_tuning best, uint32_t *out,
                     unsigned long long *counts, uint32_t ncounts, cudaStream_t st, const std::vector<uint32_t> &tiles)
{
    double tbest = time_tuning(c, reqs, best, out, counts, ncounts, st, 2);
    for (int pass = 0; pass < 2; ++pass) {
        for (int param = 0; param < 5; ++param) {
            std::vector<sieve_tuning> cand;
            const uint32_t B = 1u << best.tile_log2;
            auto push = [&](sieve_tuning t) {
                if (t.window_tiles > kScatterMaxTiles) t.window_tiles = kScatterMaxTiles;
                while (((uint64_t)t.window_tiles << t.tile_log2) > (1ull << 30)) t.window_tiles >>= 1;
                if (t.epoch_tiles < t.window_tiles) t.epoch_tiles = t.window_tiles;
                if (tuning_valid(t)) cand.push_back(t);
            };
            for (int k = 0;; ++k) {
                sieve_tuning t = best;
                if (param == 0) {
                    if (k >= (int)tiles.size()) break;
                    t.tile_log2 = tiles[k];
                    // keep the thresholds in proportion to the tile
                    const int d = (int)t.tile_log2 - (int)best.tile_log2;
                    t.coop_max = d >= 0 ? best.coop_max << d : best.coop_max >> -d;
                    t.medium_max = d >= 0 ? best.medium_max << d : best.medium_max >> -d;
                    t.window_tiles = d >= 0 ? best.window_tiles >> d : best.window_tiles << -d;
                } else if (param == 1) {
                    static const uint32_t g[] = {2, 4, 6, 8, 10, 13};
                    if (k >= 6) break;
                    t.presieve_groups = g[k];
                } else if (param == 2) {
                    if (k >= 5) break;
                    t.coop_max = B >> (5 + k);
                } else if (param == 3) {
                    static const int sh[] = {-2, -1, 0, 1, 2};
                    if (k >= 5) break;
                    t.medium_max = sh[k] >= 0 ? B << sh[k] : B >> -sh[k];
                    if (t.medium_max > (1u << 28)) continue;
                } else {
                    static const uint32_t w[] = {128, 256, 512, 1024};
                    if (k >= 4) break;
                    t.window_tiles = w[k];
                }
                push(t);
            }
            for (const sieve_tuning &t : cand) {
                if (tune_key(t) == tune_key(best)) continue;
                const double ms = time_tuning(c, reqs, t, out, counts, ncounts, st, 2);
                if (ms < tbest) {
                    tbest = ms;
                    best = t;
                }
            }
        }
    }
    return best;
}

}  // namespace

sieve_status sieve_autotune(sieve_ctx *c, uint32_t l, uint64_t f, uint64_t n, sieve_tuning *out,
                            sieve_stream stream)
try {
    if (!c || l < 5 || l > 40 || n == 0) return SIEVE_EINVAL;
    if ((((unsigned __int128)f + n) << l) > ((unsigned __int128)1 << 63)) return SIEVE_ERANGE;
    const uint64_t j0 = f << l, nbits = n << l;
    const uint64_t vlast = 2 * (j0 + nbits) - 1;
    if (isqrt_u64(vlast) > c->base_limit) return SIEVE_ERANGE;
    if (cudaSetDevice(c->device) != cudaSuccess) return SIEVE_ECUDA;
    cudaStream_t st = (cudaStream_t)stream;
    // a sample of the interval: its first 2^31 bits (or all of it)
    const uint64_t ns = std::min<uint64_t>(nbits, 1ull << 31);
    uint32_t *buf = nullptr;
    if (cudaMalloc(&buf, ns / 8 + 64) != cudaSuccess) {
        cudaGetLastError();
        return SIEVE_ENOMEM;
    }
    const uint32_t cls = tune_class(vlast);
    std::vector<ReqSpec> reqs{{j0, ns, 0, 0}};
    std::vector<uint32_t> tiles;
    for (uint32_t bt = 15; bt <= 20; ++bt)
        if ((ns >> bt) >= (uint64_t)(2 * c->nsm) || bt == 15) tiles.push_back(bt);
    const sieve_tuning best = descend(c, reqs, c->tune[cls], buf, nullptr, 0, st, tiles);
    cudaStreamSynchronize(st);
    cudaFree(buf);
    c->tune[cls] = best;
    if (out) *out = best;
    return cudaGetLastError() == cudaSuccess ? SIEVE_OK : SIEVE_ECUDA;
} catch (...) {
    return SIEVE_ENOMEM;  // host memory (or another host resource) ran out
}

sieve_status sieve_autotune_batch(sieve_ctx *c, const sieve_req *reqs, uint32_t count, uint32_t *dev_arena,
                                  uint64_t *dev_counts, sieve_tuning *out, sieve_stream stream)
try {
    if (!c || !reqs || !count || !dev_arena || !dev_counts) return SIEVE_EINVAL;
    if (cudaSetDevice(c->device) != cudaSuccess) return SIEVE_ECUDA;
    std::vector<ReqSpec> rs(count);
    std::vector<uint64_t> vl(count);
    uint64_t vmax = 0;
    for (uint32_t r = 0; r < count; ++r) {
        if (reqs[r].nbits == 0 || (reqs[r].j0 & 31) || (reqs[r].nbits & 31)) return SIEVE_EINVAL;
        const unsigned __int128 jend = (unsigned __int128)reqs[r].j0 + reqs[r].nbits;
        if (jend > ((unsigned __int128)1 << 63)) return SIEVE_ERANGE;
        vl[r] = (uint64_t)(2 * jend - 1);
        if (isqrt_u64(vl[r]) > c->base_limit) return SIEVE_ERANGE;
        rs[r] = ReqSpec{reqs[r].j0, reqs[r].nbits, reqs[r].out_word_off, r};
        vmax = std::max(vmax, vl[r]);
    }
    std::stable_sort(rs.begin(), rs.end(), [&](const ReqSpec &a, const ReqSpec &b) { return vl[a.idx] > vl[b.idx]; });
    const sieve_tuning start = c->batch_tune.tile_log2 ? c->batch_tune : c->tune[tune_class(vmax)];
    const std::vector<uint32_t> tiles{16, 17, 18, 19, 20};
    const sieve_tuning best = descend(c, rs, start, dev_arena, (unsigned long long *)dev_counts, count,
                                      (cudaStream_t)stream, tiles);
    c->batch_tune = best;
    c->plans.clear();
    if (out) *out = best;
    return cudaGetLastError() == cudaSuccess ? SIEVE_OK : SIEVE_ECUDA;
} catch (...) {
    return SIEVE_ENOMEM;  // host memory (or another host resource) ran out
}
