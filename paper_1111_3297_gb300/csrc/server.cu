// Serving: a request loop with continuous batching.
//
// One scheduler thread owns all device work of the server.  Requests wait in a
// FIFO; whenever a lane (a stream with its own scratch) is free, the scheduler
// admits requests from the head of the FIFO while their tables fit in the
// server's device arena, plans them as one batch (the batched path of
// sieve_batch), reserves the plan's two large-prime bucket pools in the same
// arena and launches it on that lane.  Tables and buckets thus share one memory
// cap: a batch is admitted only when both its tables and its buckets fit, its
// buckets return to the arena when it completes, and its tables when the client
// releases them.  Lanes run concurrently, so a
// request that arrives while others are on the GPU starts as soon as a lane and
// memory free up.  Completion is observed with cudaEventQuery (no blocking
// waits), the composite counts come back in pinned memory, and the table stays
// in the arena until the client releases it.
#include "gbsieve.h"
#include "host_internal.h"

#include <algorithm>
#include <atomic>
#include <chrono>
#include <condition_variable>
#include <deque>
#include <map>
#include <mutex>
#include <thread>
#include <vector>

using namespace gbs;

namespace {

constexpr uint64_t kGranule = 256;      // table arena granularity (bytes)
constexpr uint32_t kMaxBatch = 1024;    // requests per launched batch
constexpr uint64_t kMaxBatchBits = 1ull << 34;

// first-fit allocator over [0, size) with coalescing free list
struct Arena {
    std::map<uint64_t, uint64_t> free_;  // offset -> size
    uint64_t size = 0, used = 0;
    void init(uint64_t n) {
        size = n;
        free_.clear();
        free_[0] = n;
        used = 0;
    }
    uint64_t largest() const {
        uint64_t m = 0;
        for (const auto &kv : free_) m = std::max(m, kv.second);
        return m;
    }
    bool alloc(uint64_t n, uint64_t *off) {
        n = (n + kGranule - 1) / kGranule * kGranule;
        for (auto it = free_.begin(); it != free_.end(); ++it) {
            if (it->second >= n) {
                *off = it->first;
                const uint64_t rest = it->second - n, o = it->first;
                free_.erase(it);
                if (rest) free_[o + n] = rest;
                used += n;
                return true;
            }
        }
        return false;
    }
    void release(uint64_t off, uint64_t n) {
        n = (n + kGranule - 1) / kGranule * kGranule;
        used -= n;
        auto it = free_.emplace(off, n).first;
        auto nx = std::next(it);
        if (nx != free_.end() && it->first + it->second == nx->first) {
            it->second += nx->second;
            free_.erase(nx);
        }
        if (it != free_.begin()) {
            auto pv = std::prev(it);
            if (pv->first + pv->second == it->first) {
                pv->second += it->second;
                free_.erase(it);
            }
        }
    }
};

struct Req {
    uint64_t id, j0, nbits;
    uint64_t off = 0, bytes = 0;  // table in the arena
    uint64_t composites = 0;
    double t_submit = 0, t_admit = 0, t_done = 0;
    int status = SIEVE_OK;
    bool admitted = false;  // its table holds arena memory
    bool done = false;
};

struct Lane {
    cudaStream_t st = nullptr;
    cudaEvent_t ev = nullptr;
    Scratch scr;
    unsigned long long *d_counts = nullptr;
    unsigned long long *h_counts = nullptr;  // pinned
    int *h_err = nullptr;                    // pinned
    std::unique_ptr<Plan> plan;
    std::vector<Req *> reqs;
    bool busy = false;
    uint64_t bkt_off = 0, bkt_bytes = 0;  // the batch's bucket pools in the arena
};

// bytes of one bucket pool of `entries` slots in the arena (granule-aligned)
uint64_t pool_bytes(uint64_t entries) { return (entries * 4 + 64 + kGranule - 1) / kGranule * kGranule; }
constexpr uint64_t kMinPoolEntries = 4096;  // the planner's smallest pool

}  // namespace

struct sieve_server {
    sieve_ctx *c = nullptr;
    uint32_t *d_arena = nullptr;
    Arena arena;
    std::vector<Lane> lanes;
    std::thread th;
    std::mutex mu;
    std::condition_variable cv_work, cv_done;
    std::deque<Req *> pending;
    std::deque<Req *> done_q;
    std::map<uint64_t, Req *> live;
    uint64_t next_id = 1;
    bool stop = false;
    std::chrono::steady_clock::time_point t0;
    double now() const {
        return std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
    }
    uint64_t lane_max_entries = 0;  // largest bucket pool a lane's batch may take
    // arena releases so far; a batch rolled back for want of bucket memory blocks
    // admission until the next release (no replanning while nothing has changed)
    uint64_t mem_epoch = 0, blocked_epoch = ~0ull;
    void loop();
    int launch(Lane &L, std::vector<Req *> &batch, bool others_busy);
    void complete(Lane &L);
    bool head_fits();
};

// the head of the queue could be admitted now: its table and the smallest bucket
// pools fit in the arena at once (called with mu held)
bool sieve_server::head_fits()
{
    if (pending.empty()) return false;
    uint64_t o1 = 0, o2 = 0;
    if (!arena.alloc(pending.front()->bytes, &o1)) return false;
    const bool ok = arena.alloc(2 * pool_bytes(kMinPoolEntries), &o2);
    if (ok) arena.release(o2, 2 * pool_bytes(kMinPoolEntries));
    arena.release(o1, pending.front()->bytes);
    return ok;
}

// Returns 1 when the batch is on the GPU, 0 when it failed (its requests carry the
// error; the caller completes the lane) and -1 when its bucket pools do not fit in
// the arena now (the batch went back to the head of the queue, tables released).
int sieve_server::launch(Lane &L, std::vector<Req *> &batch, bool others_busy)
try {
    std::vector<ReqSpec> rs(batch.size());
    std::vector<uint64_t> vl(batch.size());
    uint64_t vmax = 0;
    for (size_t i = 0; i < batch.size(); ++i) {
        rs[i] = ReqSpec{batch[i]->j0, batch[i]->nbits, batch[i]->off / 4, (uint32_t)i};
        vl[i] = 2 * (batch[i]->j0 + batch[i]->nbits) - 1;
        vmax = std::max(vmax, vl[i]);
    }
    std::stable_sort(rs.begin(), rs.end(), [&](const ReqSpec &a, const ReqSpec &b) { return vl[a.idx] > vl[b.idx]; });
    const sieve_tuning t = c->batch_tune.tile_log2 ? c->batch_tune : c->tune[tune_class(vmax)];
    L.plan = build_plan(c, rs, t, lane_max_entries);
    sieve_status s = L.plan ? SIEVE_OK : SIEVE_ERANGE;
    if (!s) {
        // the plan's two bucket pools, from the arena the tables come from: as the plan
        // wants them, else the largest free block when it still holds every tile's
        // bucket (more epochs, same bits) or nothing else runs (tiles beyond the pool
        // use the backstop list), else back to the queue until memory frees up
        uint32_t max_cap = 0;
        for (const TileDesc &d : L.plan->tiles) max_cap = std::max(max_cap, d.bkt_cap);
        uint64_t entries = std::max<uint64_t>(L.plan->pool_entries, kMinPoolEntries), off = 0;
        bool got;
        {
            std::lock_guard<std::mutex> g(mu);
            got = arena.alloc(2 * pool_bytes(entries), &off);
            if (!got) {
                // pools of `fit` entries take pool_bytes(fit) <= half bytes each (granule included)
                const uint64_t half = arena.largest() / 2 / kGranule * kGranule;
                const uint64_t fit = half >= 64 + kGranule + 4 * kMinPoolEntries ? ((half - 64 - kGranule) / 4) & ~3ull : 0;
                if (fit >= kMinPoolEntries && (fit >= max_cap || !others_busy)) {
                    entries = fit;
                    got = arena.alloc(2 * pool_bytes(entries), &off);
                }
            }
            if (!got) {
                // roll the batch back: tables released, requests to the head of the queue
                for (size_t i = batch.size(); i-- > 0;) {
                    Req *r = batch[i];
                    arena.release(r->off, r->bytes);
                    r->admitted = false;
                    pending.push_front(r);
                }
                blocked_epoch = mem_epoch;
                L.plan.reset();
                return -1;
            }
        }
        L.bkt_off = off;
        L.bkt_bytes = 2 * pool_bytes(entries);
        if (entries < L.plan->pool_entries) L.plan = build_plan(c, rs, t, entries);
        L.scr.d_bkt[0] = reinterpret_cast<uint32_t *>(reinterpret_cast<char *>(d_arena) + off);
        L.scr.d_bkt[1] = reinterpret_cast<uint32_t *>(reinterpret_cast<char *>(d_arena) + off + pool_bytes(entries));
        L.scr.bkt_bytes[0] = L.scr.bkt_bytes[1] = pool_bytes(entries);
        L.scr.pool_entries = entries;
        if (!L.plan) s = SIEVE_ERANGE;
    }
    Plan *P = L.plan.get();
    if (!s) s = scratch_ensure(L.scr, P->pool_entries, P->max_epoch_tiles, P->carry_entries);
    if (!s) s = upload_plan(c, P, L.st);
    if (!s) s = enqueue_plan(c, L.scr, P, d_arena, L.d_counts, (uint32_t)batch.size(), L.st);
    if (!s && cudaMemcpyAsync(L.h_counts, L.d_counts, batch.size() * 8, cudaMemcpyDeviceToHost, L.st) != cudaSuccess)
        s = SIEVE_ECUDA;
    if (!s && cudaMemcpyAsync(L.h_err, L.scr.d_err, 4, cudaMemcpyDeviceToHost, L.st) != cudaSuccess) s = SIEVE_ECUDA;
    if (!s && cudaMemsetAsync(L.scr.d_err, 0, 4, L.st) != cudaSuccess) s = SIEVE_ECUDA;
    if (!s && cudaEventRecord(L.ev, L.st) != cudaSuccess) s = SIEVE_ECUDA;
    L.reqs = batch;
    L.busy = true;
    if (s) {
        // nothing (more) will run for these requests: finish them with the error
        cudaStreamSynchronize(L.st);
        for (Req *r : L.reqs) r->status = s;
        *L.h_err = 0;
        return 0;
    }
    return 1;
} catch (...) {
    // host memory ran out while planning or enqueueing (this runs on the server's
    // thread, which an escaping exception would end): wait for whatever was
    // enqueued, then finish the batch with the error
    cudaStreamSynchronize(L.st);
    L.reqs = batch;
    L.busy = true;
    for (Req *r : L.reqs) r->status = SIEVE_ENOMEM;
    *L.h_err = 0;
    return 0;
}

void sieve_server::complete(Lane &L)
{
    const double t = now();
    const int err = *L.h_err;
    std::lock_guard<std::mutex> g(mu);
    for (size_t i = 0; i < L.reqs.size(); ++i) {
        Req *r = L.reqs[i];
        if (r->status == SIEVE_OK) {
            r->composites = L.h_counts[i];
            if (err) r->status = (err & kErrTimeout) ? SIEVE_ETIMEOUT : SIEVE_EOVERFLOW;
        }
        r->t_done = t;
        r->done = true;
        done_q.push_back(r);
    }
    L.reqs.clear();
    L.plan.reset();
    if (L.bkt_bytes) arena.release(L.bkt_off, L.bkt_bytes), ++mem_epoch;  // the batch's buckets return
    L.bkt_bytes = 0;
    L.scr.d_bkt[0] = L.scr.d_bkt[1] = nullptr;
    L.scr.bkt_bytes[0] = L.scr.bkt_bytes[1] = 0;
    L.busy = false;
    cv_done.notify_all();
}

void sieve_server::loop()
{
    cudaSetDevice(c->device);
    for (;;) {
        // 1. retire lanes whose work finished
        for (Lane &L : lanes) {
            if (!L.busy) continue;
            const cudaError_t q = cudaEventQuery(L.ev);
            if (q == cudaSuccess) {
                complete(L);
            } else if (q != cudaErrorNotReady) {
                for (Req *r : L.reqs) r->status = SIEVE_ECUDA;
                *L.h_err = 0;
                complete(L);
            }
        }
        // 2. admit from the head of the queue onto free lanes
        bool launched = false;
        for (Lane &L : lanes) {
            if (L.busy) continue;
            std::vector<Req *> batch;
            {
                std::lock_guard<std::mutex> g(mu);
                if (blocked_epoch == mem_epoch) break;  // nothing released since the last rollback
                uint64_t bits = 0;
                while (!pending.empty() && batch.size() < kMaxBatch && bits < kMaxBatchBits) {
                    Req *r = pending.front();
                    if (!arena.alloc(r->bytes, &r->off)) break;  // wait for memory
                    r->admitted = true;
                    pending.pop_front();
                    r->t_admit = now();
                    bits += r->nbits;
                    batch.push_back(r);
                }
            }
            if (batch.empty()) break;
            bool others = false;
            for (Lane &M : lanes) others |= (&M != &L) && M.busy;
            const int r = launch(L, batch, others);
            if (r < 0) break;  // buckets do not fit now: wait for a batch to finish
            if (r == 0) complete(L);
            launched = true;
        }
        // 3. sleep until new work or a short poll interval
        std::unique_lock<std::mutex> g(mu);
        bool any_busy = false;
        for (Lane &L : lanes) any_busy |= L.busy;
        if (stop && !any_busy) {
            if (pending.empty()) break;
            if (!launched) {
                // stopping, nothing in flight, and the head of the queue did not fit
                if (head_fits()) {
                    blocked_epoch = ~0ull;  // memory was released meanwhile: admit on the next pass
                    continue;
                }
                // only the client's release of held tables could make room, so the
                // queued requests end now instead of holding destroy forever
                const double t = now();
                for (Req *r : pending) {
                    r->status = SIEVE_EBUSY;
                    r->t_done = t;
                    r->done = true;
                    done_q.push_back(r);
                }
                pending.clear();
                cv_done.notify_all();
                break;
            }
        }
        if (!launched) {
            if (any_busy)
                cv_work.wait_for(g, std::chrono::microseconds(50));
            else
                cv_work.wait_for(g, std::chrono::milliseconds(2), [&] {
                    return stop || (!pending.empty() && blocked_epoch != mem_epoch);
                });
        }
    }
}

sieve_status sieve_server_create(sieve_ctx *c, size_t mem_cap, uint32_t max_inflight, sieve_server **out)
try {
    if (!c || !out || max_inflight == 0 || max_inflight > 16 || mem_cap < ((size_t)256 << 20)) return SIEVE_EINVAL;
    if (cudaSetDevice(c->device) != cudaSuccess) return SIEVE_ECUDA;
    std::unique_ptr<sieve_server> S(new sieve_server());
    S->c = c;
    S->t0 = std::chrono::steady_clock::now();
    // one arena of mem_cap bytes holds the admitted requests' tables and the running
    // batches' bucket pools; a batch's two pools hold at most lane_pool bytes together
    // (a quarter of the cap shared by the lanes, at most 4 GiB), and less when the plan
    // needs less
    const uint64_t lane_pool = std::min<uint64_t>((uint64_t)4 << 30, mem_cap / 4 / max_inflight);
    S->lane_max_entries = lane_pool / 8;
    const uint64_t arena = mem_cap;
    if (cudaMalloc(&S->d_arena, arena) != cudaSuccess) {
        cudaGetLastError();
        return SIEVE_ENOMEM;
    }
    S->arena.init(arena);
    S->lanes.resize(max_inflight);
    for (Lane &L : S->lanes) {
        if (cudaStreamCreateWithFlags(&L.st, cudaStreamNonBlocking) != cudaSuccess ||
            cudaEventCreateWithFlags(&L.ev, cudaEventDisableTiming) != cudaSuccess ||
            cudaMalloc(&L.d_counts, kMaxBatch * 8) != cudaSuccess ||
            cudaMallocHost(&L.h_counts, kMaxBatch * 8) != cudaSuccess ||
            cudaMallocHost(&L.h_err, 16) != cudaSuccess) {
            cudaGetLastError();
            sieve_server_destroy(S.release());
            return SIEVE_ENOMEM;
        }
        *L.h_err = 0;
        L.scr.ext_pools = true;  // set before anything can free the scratch
        if (scratch_init(L.scr, S->lane_max_entries, 1u << 20) != SIEVE_OK) {
            sieve_server_destroy(S.release());
            return SIEVE_ENOMEM;
        }
    }
    sieve_server *raw = S.release();
    raw->th = std::thread([raw] { raw->loop(); });
    *out = raw;
    return SIEVE_OK;
} catch (...) {
    return SIEVE_ENOMEM;  // host memory (or another host resource) ran out
}

sieve_status sieve_server_submit(sieve_server *S, uint64_t j0, uint64_t nbits, uint64_t *id)
try {
    if (!S || !id) return SIEVE_EINVAL;
    uint64_t vlast;
    sieve_status s = check_range(S->c, j0, nbits, &vlast);
    if (s) return s;
    // never admissible: its table and the smallest bucket pools exceed the whole arena
    if (nbits / 8 + kGranule + 2 * pool_bytes(kMinPoolEntries) > S->arena.size) return SIEVE_ENOMEM;
    Req *r = new Req();
    r->j0 = j0;
    r->nbits = nbits;
    r->bytes = nbits / 8;
    {
        std::lock_guard<std::mutex> g(S->mu);
        if (S->stop) {
            delete r;
            return SIEVE_EBUSY;
        }
        r->id = S->next_id++;
        r->t_submit = S->now();
        S->pending.push_back(r);
        S->live[r->id] = r;
    }
    *id = r->id;
    S->cv_work.notify_one();
    return SIEVE_OK;
} catch (...) {
    return SIEVE_ENOMEM;  // host memory (or another host resource) ran out
}

sieve_status sieve_server_poll(sieve_server *S, sieve_result *out, uint32_t max, uint32_t *n, uint32_t timeout_ms)
try {
    if (!S || !n || (max && !out)) return SIEVE_EINVAL;
    *n = 0;
    std::unique_lock<std::mutex> g(S->mu);
    if (S->done_q.empty() && timeout_ms)
        S->cv_done.wait_for(g, std::chrono::milliseconds(timeout_ms), [&] { return !S->done_q.empty(); });
    while (*n < max && !S->done_q.empty()) {
        Req *r = S->done_q.front();
        S->done_q.pop_front();
        sieve_result &o = out[(*n)++];
        o.id = r->id;
        o.j0 = r->j0;
        o.nbits = r->nbits;
        o.composites = r->composites;
        o.dev_bits = S->d_arena + r->off / 4;
        o.t_submit = r->t_submit;
        o.t_admit = r->t_admit;
        o.t_done = r->t_done;
        o.status = r->status;
    }
    return SIEVE_OK;
} catch (...) {
    return SIEVE_ENOMEM;  // host memory (or another host resource) ran out
}

sieve_status sieve_server_release(sieve_server *S, uint64_t id)
try {
    if (!S) return SIEVE_EINVAL;
    std::lock_guard<std::mutex> g(S->mu);
    auto it = S->live.find(id);
    if (it == S->live.end() || !it->second->done) return SIEVE_EINVAL;
    if (it->second->admitted) S->arena.release(it->second->off, it->second->bytes), ++S->mem_epoch;
    delete it->second;
    S->live.erase(it);
    S->cv_work.notify_one();
    return SIEVE_OK;
} catch (...) {
    return SIEVE_ENOMEM;  // host memory (or another host resource) ran out
}

double sieve_server_now(sieve_server *S) { return S ? S->now() : 0.0; }

void sieve_server_destroy(sieve_server *S)
{
    if (!S) return;
    {
        std::lock_guard<std::mutex> g(S->mu);
        S->stop = true;
    }
    S->cv_work.notify_all();
    if (S->th.joinable()) S->th.join();
    cudaSetDevice(S->c->device);
    for (Lane &L : S->lanes) {
        if (L.st) cudaStreamSynchronize(L.st);
        L.plan.reset();
        scratch_free(L.scr);
        if (L.st) cudaStreamDestroy(L.st);
        if (L.ev) cudaEventDestroy(L.ev);
        if (L.d_counts) cudaFree(L.d_counts);
        if (L.h_counts) cudaFreeHost(L.h_counts);
        if (L.h_err) cudaFreeHost(L.h_err);
    }
    for (auto &kv : S->live) delete kv.second;
    if (S->d_arena) cudaFree(S->d_arena);
    delete S;
}
