/*
 * gbsieve — odd-only segmented sieve of Eratosthenes on NVIDIA GB300 (sm_103a).
 *
 * C ABI of libgbsieve.so.  Plain pointers and sizes only.  Device pointers are
 * CUDA device addresses (e.g. from cudaMalloc or a torch CUDA tensor); host
 * pointers are ordinary process memory.  Streams are cudaStream_t values
 * (0 = the legacy default stream).  Every call that takes a stream enqueues its
 * device work asynchronously on that stream unless the comment says it waits.
 *
 * The table (Jarai & Vatai, "Cache optimized linear sieve", Definition "Sieve
 * table, Segments", Sec. 1.3): for parameters l, f, n (Sec. 1.2.1) it has
 * n*2^l bits; bit j stands for the odd number 2(f*2^l + j) + 1 and is 1 exactly
 * when that number is composite (so 1 and every prime read 0).  The numbers
 * covered are u = f*2^(l+1)+1 .. v = (f+n)*2^(l+1).
 * Layout: bit j is bit (j % 32) of 32-bit word j / 32 (least significant bit
 * first), words consecutive in memory.
 *
 * Errors: argument and allocation errors are returned at once.  An error raised
 * on the device (a bucket overflow beyond the backstop) is recorded in the
 * context and returned by the next call that waits on the stream (sieve_count,
 * sieve_sync, sieve_segments_host).  A call whose work would exceed 2^31 on-chip
 * tiles returns SIEVE_ERANGE; host allocation failures return SIEVE_ENOMEM (no C++
 * exception crosses this interface).  No kernel waits on another CTA or launch, so
 * no device wait can hang.  Functions are not thread-safe on one context, except
 * the server functions, which lock.  Calls on one context may be issued on different
 * streams: the context's device work runs one call after another (each starts after
 * the previous call's), since all of it shares the context's bucket pools.
 */
#ifndef GBSIEVE_H
#define GBSIEVE_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct CUstream_st *sieve_stream; /* same type as cudaStream_t */
typedef struct sieve_ctx sieve_ctx;

typedef enum {
    SIEVE_OK = 0,
    SIEVE_EINVAL = 1,    /* bad argument (null pointer, l out of range, n = 0, misaligned) */
    SIEVE_ERANGE = 2,    /* numbers beyond 2^64, or sqrt(v) beyond the context's base */
    SIEVE_ENOMEM = 3,    /* device or host allocation failed / over the memory budget */
    SIEVE_ECUDA = 4,     /* a CUDA runtime call failed */
    SIEVE_ETIMEOUT = 5,  /* a bounded wait ran out (reserved: no current call reports it) */
    SIEVE_EBUSY = 6,     /* server queue full / resource in use */
    SIEVE_EOVERFLOW = 7  /* large-prime bucket overflow beyond the backstop list */
} sieve_status;

/* Text for a status code (static storage). */
const char *sieve_strerror(sieve_status s);

/* For SIEVE_ECUDA: the failed CUDA runtime call and its error text, as seen by the
 * last failing call on this host thread ("" if none).  Storage belongs to the
 * library, per thread, until that thread's next failing call. */
const char *sieve_last_cuda_error(void);

/*
 * Create a context on CUDA device `device`, able to sieve any interval whose
 * largest number is <= max_v.  Builds the base of Sec. 1.4 (Definition "base":
 * the odd primes p <= sqrt(max_v)) on the device and keeps it resident with one
 * 64-bit reduction constant per prime.  mem_budget bounds the device memory the
 * context uses for large-prime buckets (0 = 16 GiB; otherwise at least 64 MiB,
 * else SIEVE_EINVAL; split into two pools of mem_budget / 8 slots).
 * Waits for the device.
 * On success *ctx owns all its device memory until sieve_destroy.
 */
sieve_status sieve_init(sieve_ctx **ctx, int device, uint64_t max_v, size_t mem_budget);

/* Free the context and everything it owns.  NULL is ignored. */
void sieve_destroy(sieve_ctx *ctx);

/*
 * The sieve table for (l, f, n) (Sec. 1.2.1, Sec. 1.3) into caller-owned device
 * memory dev_bits of n*2^(l-5) uint32 words (16-byte aligned).  5 <= l <= 40,
 * n >= 1, (f+n)*2^(l+1) < 2^64, and isqrt(v-1) within the context's base, else
 * SIEVE_EINVAL / SIEVE_ERANGE.  Asynchronous on `stream`; dev_bits must stay
 * valid until the stream reaches the work.  The segment size the device uses
 * internally is the autotuner's choice; the bits do not depend on it.
 */
sieve_status sieve_segments(sieve_ctx *ctx, uint32_t l, uint64_t f, uint64_t n,
                            uint32_t *dev_bits, sieve_stream stream);

/*
 * As sieve_segments, with f chosen from the midpoint M = mant * 10^exp10 as in
 * Sec. 1.2.1 (the midpoint input): f = max(0, floor(M / 2^(l+1)) - floor(n/2)).
 */
sieve_status sieve_f_from_midpoint(uint32_t l, uint64_t n, uint64_t mant, uint32_t exp10,
                                   uint64_t *f_out);
sieve_status sieve_segments_midpoint(sieve_ctx *ctx, uint32_t l, uint64_t mant, uint32_t exp10,
                                     uint64_t n, uint32_t *dev_bits, sieve_stream stream);

/*
 * Prime and twin-prime counts per segment, without writing the table: a consumer of
 * the sieve table fused into the segment kernel (Sec. 5 names such uses of the table;
 * Definition "Sieve table, Segments", Sec. 1.3, fixes the segments).  Sieves the same
 * interval as sieve_segments(l, f, n) and, for each segment t < n (the 2^l odd numbers
 * m = 2(f*2^l + t*2^l + j) + 1, 0 <= j < 2^l), writes to caller-owned device memory
 *   dev_primes[t]  the number of primes m in segment t (1 is not a prime);
 *   dev_twins[t]   the number of twin pairs (m, m + 2), both prime, with m in segment t
 *                  and m + 2 inside the interval (NULL: not counted).
 * Both arrays are uint64_t[n], 8-byte aligned; they are overwritten (not accumulated),
 * asynchronously on `stream`.  The sum of dev_primes is the interval's prime count.
 * Requires 12 <= l <= 40 (segments of at least 4096 bits); otherwise as sieve_segments
 * (SIEVE_EINVAL, SIEVE_ERANGE; device errors at the next waiting call).  The call keeps
 * a plan per (interval, output pointers), like sieve_segments.
 */
sieve_status sieve_count_segments(sieve_ctx *ctx, uint32_t l, uint64_t f, uint64_t n,
                                  uint64_t *dev_primes, uint64_t *dev_twins, sieve_stream stream);

/*
 * Goldbach search on a finished table (Sec. 5: verifying the Goldbach conjecture is
 * the use the authors built the sieve for).  dev_bits holds a table in the layout of
 * sieve_segments: bit j (word j/32, bit j%32) stands for the odd number 2(j0 + j) + 1,
 * 0 for primes (and the number 1), j < nbits (nbits % 32 == 0).  For every even
 * N = n_lo + 2i, 0 <= i < count (n_lo even, >= 4), the device finds the smallest odd
 * prime p <= p_max with N - p prime by reading the table, trying p = 3, 5, 7, ... in
 * order.  Per window w of 2^win_log2 consecutive i (5 <= win_log2 <= 32) it writes
 * dev_windows[w] (caller-owned device memory, ceil(count / 2^win_log2) entries, 8-byte
 * aligned, overwritten):
 *   key       (largest minimal p in the window) << 32 | (2^32 - 1 - k), k the offset
 *             in the window of the first N attaining it; 0 when no N of the window
 *             has such a p;
 *   failures  even numbers of the window with no odd prime p <= p_max for which
 *             N - p is prime (within p_max: a candidate counterexample, or p_max too
 *             small).
 * The table must hold N - 3 for the largest N, and, unless j0 == 0, N - p_max for the
 * smallest N (SIEVE_ERANGE otherwise); p_max must not exceed the context's base limit
 * (the primes tried are the context's resident base primes).  Asynchronous on
 * `stream`; the table must be complete on that stream.  SIEVE_EINVAL for null or
 * misaligned pointers, odd n_lo, count 0 or win_log2 out of range.
 */
typedef struct {
    uint64_t key;
    uint64_t failures;
} sieve_goldbach_window;
sieve_status sieve_goldbach(sieve_ctx *ctx, const uint32_t *dev_bits, uint64_t j0, uint64_t nbits,
                            uint64_t n_lo, uint64_t count, uint32_t p_max, uint32_t win_log2,
                            sieve_goldbach_window *dev_windows, sieve_stream stream);

/*
 * End-to-end form of sieve_segments: the table lands in caller-owned HOST memory
 * host_bits (n*2^(l-5) words; pinned memory copies fastest).  The context sieves
 * it in epochs of at most 2^30 bits into a two-slot device ring and copies each
 * slot back while the next epochs are sieved (device memory: two epochs).  Waits
 * until the table is in host_bits.
 */
sieve_status sieve_segments_host(sieve_ctx *ctx, uint32_t l, uint64_t f, uint64_t n,
                                 uint32_t *host_bits, sieve_stream stream);

/*
 * Number of 1 bits (composites) in the first nbits bits of the device table
 * dev_bits (nbits % 32 == 0).  Waits for `stream` and writes *host_count.
 * Primes in the table's range = nbits - composites - (1 if the table starts at
 * the number 1, since 1 is neither): the prime count of the interval that the table of
 * Definition "Sieve table, Segments" (Sec. 1.3) encodes.  SIEVE_EINVAL for a null
 * pointer or nbits not a multiple of 32; a device error recorded since the last wait
 * is returned here (the count is then not meaningful).
 */
sieve_status sieve_count(sieve_ctx *ctx, const uint32_t *dev_bits, uint64_t nbits,
                         uint64_t *host_count, sieve_stream stream);

/*
 * Composite count without any allocation (the paper has no counterpart; this is a
 * service for callers that cannot allocate device memory: code whose device
 * memory is owned by another framework's pool, and latency-critical code that
 * must not risk the implicit device synchronisation of cudaMalloc/cudaFree).
 * Needs no context.  Counts the 1 bits of the first nbits bits of dev_bits
 * (nbits % 32 == 0, at most SIEVE_NOALLOC_MAX_BITS, else SIEVE_ERANGE) on the
 * current device and writes the count to the caller-owned device word
 * *dev_count, asynchronously on `stream`.  Its only scratch is a fixed 512 KB
 * array of partial counts inside the library, which every GPU that loads the
 * library holds until the process exits.  The first call on a device resolves
 * that array's device address (a one-time set-up with the device current); make
 * the first call on each device before any stream capture.  The address is kept
 * per device together with the id of the context it belongs to; after a device
 * reset the next call resolves it again.  All calls share the array and each
 * overwrites the entries it uses, so calls that overlap on the GPU (e.g. on two
 * streams at once) race and must be ordered by the caller.  SIEVE_ECUDA names the
 * failed step in sieve_last_cuda_error(); an error already pending on the calling
 * thread is reported that way too, without launching, and is not cleared.
 */
#define SIEVE_NOALLOC_MAX_BITS (1ull << 37)
sieve_status sieve_count_noalloc(const uint32_t *dev_bits, uint64_t nbits, uint64_t *dev_count,
                                 sieve_stream stream);

/*
 * Streaming of consecutive intervals (enable = 1; 0 turns it off).  A long range sieved
 * as consecutive calls of sieve_segments (or sieve_segments_host, sieve_count_segments),
 * each starting where the previous one ended, is the paper's own mode of work (Sec. 2.4:
 * segments in order, each large prime's next hit carried along, Sec. 2.3).  With
 * streaming on, every single-interval call keeps its large primes' next hits after its
 * last segment in the context, and a call that starts exactly where the previous one
 * ended, with the same tuning class choices (large-prime bound and wheel), continues
 * from them instead of computing each large prime's first hit again; primes the new
 * interval adds take first hits as usual.  The bits are the same either way.  Any other
 * call that runs device work on the context (a batch, an interval elsewhere, a tuning
 * run) ends the continuation; so does turning streaming on or off.  Calls must come in
 * order on one stream (or be ordered by the caller).  While streaming is on, single
 * intervals run without CUDA-graph replay.
 */
sieve_status sieve_set_streaming(sieve_ctx *ctx, int enable);

/* Wait for `stream` and report any device-side error recorded since the last wait. */
sieve_status sieve_sync(sieve_ctx *ctx, sieve_stream stream);

/*
 * Batched form: `count` independent interval requests in one launch sequence.
 * Request r covers absolute bit indices j0 .. j0+nbits-1 (numbers 2J+1), with
 * j0 and nbits multiples of 32 and nbits >= 32; its table goes to
 * dev_arena + out_word_off (words, caller-owned device memory) and its composite
 * count to dev_counts[r] (uint64, overwritten).  Bits are those of
 * sieve_segments for the same numbers.  Asynchronous; host_reqs may be reused
 * when the call returns.  The launch sequence is captured in a CUDA graph that
 * is replayed when the same request list is submitted again.
 */
typedef struct {
    uint64_t j0;
    uint64_t nbits;
    uint64_t out_word_off;
} sieve_req;
/* Errors: SIEVE_EINVAL (null pointers with count > 0, dev_arena not 4-byte aligned, a
 * request not word aligned or empty), SIEVE_ERANGE (a request beyond 2^64 or the context's base, or more than 2^31
 * tiles in all); nothing is enqueued then.  Requests may not overlap in the arena. */

sieve_status sieve_batch(sieve_ctx *ctx, const sieve_req *host_reqs, uint32_t count,
                         uint32_t *dev_arena, uint64_t *dev_counts, sieve_stream stream);

/*
 * Tuning of the device path (none of it changes the bits); sieve_set_tuning
 * returns SIEVE_EINVAL outside these ranges:
 *   tile_log2     on-chip segment size 2^tile_log2 bits (12..21), one CTA per tile up
 *                 to 2^20; 21 holds a segment across a cluster of two CTAs (distributed
 *                 shared memory, one interval only: batches, servers and the count
 *                 mode take 2^20; measured slower than 20 on GB300, hence opt-in);
 *   presieve_groups  how many small-prime pattern groups pre-sieve a tile
 *                 (1..13; group 1 = {3,5,7,11,13}, up to 127 with 13 groups);
 *   coop_max      primes up to this are struck by a whole warp, 32 multiples at a
 *                 time (the smallest of them, up to 2^tile_log2 / (240 * warps), by
 *                 the whole CTA); larger ones by one thread each;
 *   medium_max    primes up to this (at most 2^28) are struck inside the tile
 *                 kernel; larger primes go through the large-prime buckets;
 *   window_tiles  tiles per scatter group (the flush domain of the bucket
 *                 scatter), 1..1024, at most 2^30 bits;
 *   epoch_tiles   tiles whose buckets one scatter launch fills (window_tiles..65535;
 *                 an epoch also ends where the bucket pool is full).
 */
typedef struct {
    uint32_t tile_log2;
    uint32_t presieve_groups;
    uint32_t coop_max;
    uint32_t medium_max;
    uint32_t window_tiles;
    uint32_t epoch_tiles;
} sieve_tuning;

/* Tuning classes: by the magnitude of the interval's largest number.  cls must be
 * below SIEVE_TUNE_CLASSES (else SIEVE_EINVAL). */
#define SIEVE_TUNE_CLASSES 4 /* < 2^40, < 2^50, < 2^56, >= 2^56 */
sieve_status sieve_get_tuning(sieve_ctx *ctx, uint32_t cls, sieve_tuning *out);
/* Replaces the tuning of class cls (SIEVE_EINVAL if out of range); it also drops a
 * tuning sieve_autotune_batch stored, so batches follow the classes again. */
sieve_status sieve_set_tuning(sieve_ctx *ctx, uint32_t cls, const sieve_tuning *in);

/*
 * Autotune the class that (l, f, n) falls in: time candidate tunings on a
 * sample of that interval (writing scratch device memory the context owns),
 * keep the fastest in the context and return it in *out.  Waits for the device.
 */
sieve_status sieve_autotune(sieve_ctx *ctx, uint32_t l, uint64_t f, uint64_t n,
                            sieve_tuning *out, sieve_stream stream);

/*
 * Autotune the batched form on a request list (as for sieve_batch): time candidate
 * tile sizes (2^16..2^20 bits), medium/large thresholds and windows on the
 * actual requests, writing dev_arena / dev_counts as sieve_batch would; the
 * fastest becomes the tuning sieve_batch uses from then on (until the next
 * sieve_set_tuning).  Waits for the device.
 */
sieve_status sieve_autotune_batch(sieve_ctx *ctx, const sieve_req *host_reqs, uint32_t count,
                                  uint32_t *dev_arena, uint64_t *dev_counts, sieve_tuning *out,
                                  sieve_stream stream);

/* The base of Sec. 1.4 (Definition "base") resident in the context: *dev_primes
 * receives a device pointer to the odd primes 3 <= p <= *limit in ascending order
 * (owned by the context, valid until sieve_destroy; do not write), *count their
 * number, *limit = isqrt of the context's max_v (capped at 2^32 - 1).  Any of the
 * three pointers may be NULL. */
sieve_status sieve_base_info(sieve_ctx *ctx, const uint32_t **dev_primes, uint64_t *count,
                             uint64_t *limit);

/*
 * Per-kernel timing of the device work of later calls, by CUDA events on the
 * stream each kernel runs on (enable = 1 turns it on, 0 off; 2 also runs the
 * scatter and tile launches of a plan on one stream, one after the other, so that
 * each kernel's time is its own rather than shared with the other overlapping
 * it).  sieve_profile_read waits for the stream and returns, per kernel kind, the
 * launches and the summed milliseconds since the last read, plus work counters.
 */
typedef struct {
    uint64_t launches[8];    /* by kind, see SIEVE_K_* */
    double ms[8];
    uint64_t tiles;          /* tiles sieved */
    uint64_t bits;           /* table bits written */
    uint64_t large_hits;     /* bucket entries emitted (large-prime hits) */
    uint64_t medium_marks;   /* estimated in-tile marks by medium primes */
    uint64_t prime_reads;    /* (prime, scatter unit) visits in the scatter */
    uint64_t continued;      /* large primes that continued from the previous interval's
                                state instead of taking a first hit (streaming) */
    uint64_t state_writes;   /* 8-byte state words the single-interval scatter wrote back:
                                one per prime and scatter group, except in the interval's
                                last group when the interval is not streamed */
} sieve_profile;
#define SIEVE_K_TILE 0
#define SIEVE_K_SCATTER 1
#define SIEVE_K_COUNT 2
#define SIEVE_K_RESET 3
#define SIEVE_K_COPY 4
sieve_status sieve_profile_enable(sieve_ctx *ctx, int enable);
sieve_status sieve_profile_read(sieve_ctx *ctx, sieve_profile *out, sieve_stream stream);

/*
 * Micro-benchmark of the device's shared-memory atomic OR rate (the denominator
 * of the in-tile marking roofline): every SM runs CTAs that OR single bits into
 * random words of a shared array; returns atomics per second over the whole GPU.
 * Waits for the device.
 */
sieve_status sieve_probe_smem_atomics(int device, double *atomics_per_s);

/*
 * Micro-benchmark of distributed shared memory (thread-block clusters; the cost that
 * decides whether a segment larger than one SM's shared memory pays, Sec. 2.2: a larger
 * segment leaves fewer primes large).  Clusters of cluster_size CTAs (2, 4 or 8) of
 * 1024 threads and 128 KB each, as many as fit at once, OR single bits into
 * conflict-free words through the cluster window: of their own CTA (peer = 0) or of
 * the next rank in the cluster (peer = 1).  Returns ORs per second over the whole GPU
 * and the CTAs that ran (*ctas).  Waits for the device.
 */
sieve_status sieve_probe_dsmem_atomics(int device, uint32_t cluster_size, int peer, double *atomics_per_s,
                                       uint32_t *ctas);

/*
 * Planner inspection on the host, without a device.  Builds the plan sieve_batch
 * builds for the requests `reqs` (rules as for sieve_batch): the work
 * decomposition of Sec. 1.3 (segments = tiles) and Sec. 2.2 (large primes in
 * per-tile buckets), and reports its shape.  A single request with tuning t is
 * the plan sieve_segments runs for that interval with that tuning.
 *   host_primes  the base: all odd primes 3 <= p <= isqrt(max_v), ascending (host
 *                memory, nprimes of them; the caller vouches for completeness,
 *                only order, oddness and the bound are checked);
 *   nsm          SMs to plan chunks for (1..1024);
 *   t            tuning (ranges as for sieve_set_tuning); NULL = what a fresh context
 *                takes: for one request sieve_segments' choice (the class default,
 *                with smaller tiles when the interval has fewer than 4 per SM),
 *                else the default of the largest request's class;
 *   pool_entries bucket slots per epoch (>= 4096, at most 2^32 - 2^22).
 *                sieve_init's contexts have mem_budget / 8 of them.
 * *info receives the counts.  tiles / groups / chunks may each be NULL; otherwise
 * they receive the first max_* records (the counts in *info say how many exist).
 * Records hold base-prime indices (0 = the prime 3) and bit indices as in sieve_req.
 * Caller owns every buffer; nothing is retained.  Errors: SIEVE_EINVAL (null info,
 * bad primes, tuning or sizes; request rules of sieve_batch), SIEVE_ERANGE (a
 * request beyond max_v or 2^64).
 */
typedef struct {
    uint64_t ntiles, ngroups, nepochs, nchunks, nunits;
    uint64_t bits;             /* table bits of all tiles */
    uint64_t pool_entries;     /* bucket slots of the largest epoch */
    uint64_t carry_entries;    /* carried large-prime state slots */
    uint32_t max_epoch_tiles;
    uint32_t big_wheel;        /* 1: large primes on the mod-15015 wheel, 0: mod 15 */
    uint32_t run_scatter;      /* 1: one state word per large prime for the interval */
    uint32_t carried_groups;   /* groups whose large-prime state comes from the previous one */
    uint32_t med_lo, blk_hi, coop_hi, large_lo; /* base-index bounds of the striking phases */
    double expected_large_hits;
} sieve_plan_info;

typedef struct {
    uint64_t j0;          /* first bit index */
    uint64_t out_word;    /* output word offset */
    uint64_t bkt_off;     /* bucket offset in its epoch's pool */
    uint32_t len;         /* bits */
    uint32_t req;         /* request index */
    uint32_t epoch;
    uint32_t group;       /* scatter group, UINT32_MAX when the tile has no large primes */
    uint32_t bkt_cap;     /* bucket slots */
    uint32_t med_hi;      /* medium primes are base indices [med_lo, med_hi) */
} sieve_plan_tile;

typedef struct {
    uint32_t epoch, tile0, ntiles;  /* tiles [tile0, tile0 + ntiles), plan-wide indices */
    uint32_t nunits;                /* scatter units (runs of one request) */
    uint32_t p_lo, p_hi;            /* large primes, base indices [p_lo, p_hi) */
    uint32_t carry_in, carry_out;
} sieve_plan_group;

typedef struct {
    uint32_t epoch, p_lo, p_hi;     /* one scatter CTA: base indices [p_lo, p_hi) */
} sieve_plan_chunk;

sieve_status sieve_plan_describe(const uint32_t *host_primes, uint64_t nprimes, uint64_t max_v, uint32_t nsm,
                                 const sieve_req *reqs, uint32_t count, const sieve_tuning *t,
                                 uint64_t pool_entries, sieve_plan_info *info,
                                 sieve_plan_tile *tiles, uint64_t max_tiles,
                                 sieve_plan_group *groups, uint64_t max_groups,
                                 sieve_plan_chunk *chunks, uint64_t max_chunks);

/*
 * Serving: a request loop with continuous batching.  Requests are submitted
 * from any host thread; a scheduler thread admits them while the in-flight
 * tables plus bucket memory stay within mem_cap bytes and at most max_inflight
 * batches run, groups the admitted ones into a batch and launches it on the
 * next of its streams, so that batches overlap on the device.  Base primes and
 * bucket pools stay resident.  Results are read with sieve_server_poll: the
 * composite count, a device pointer to the request's table inside the server's
 * memory (valid until sieve_server_release) and the completion time.
 * mem_cap >= 256 MiB and 1 <= max_inflight <= 16, else SIEVE_EINVAL.  Each batch
 * runs on a scratch of its own (two bucket pools of mem_cap / (32 * max_inflight)
 * slots, at most 2^29), so the server's work never waits on the context's other
 * calls. The scheduler reads the context's tunings, so sieve_set_tuning and
 * the autotuners must not run while a server on the context is live.
 */
typedef struct sieve_server sieve_server;
typedef struct {
    uint64_t id;            /* as returned by submit */
    uint64_t j0, nbits;
    uint64_t composites;
    const uint32_t *dev_bits;
    double t_submit, t_admit, t_done; /* seconds on the server's monotonic clock */
    int status;             /* sieve_status of the request */
} sieve_result;

sieve_status sieve_server_create(sieve_ctx *ctx, size_t mem_cap, uint32_t max_inflight,
                                 sieve_server **srv);
/* Queue one request (bit indices j0 .. j0+nbits-1, word aligned as for sieve_batch);
 * *id identifies it in the results.  SIEVE_EINVAL / SIEVE_ERANGE as for sieve_batch,
 * SIEVE_ENOMEM when its table could never fit the server's memory, SIEVE_EBUSY once
 * the server is stopping. */
sieve_status sieve_server_submit(sieve_server *srv, uint64_t j0, uint64_t nbits, uint64_t *id);
/* Up to max results that completed since the last poll; *n receives how many.
 * timeout_ms > 0 waits (bounded) for at least one. */
sieve_status sieve_server_poll(sieve_server *srv, sieve_result *out, uint32_t max, uint32_t *n,
                               uint32_t timeout_ms);
/* Return a polled result's table memory to the server (SIEVE_EINVAL for an id that is
 * unknown, already released or not yet completed). */
sieve_status sieve_server_release(sieve_server *srv, uint64_t id);
/* Seconds on the server's monotonic clock (the clock of the result timestamps). */
double sieve_server_now(sieve_server *srv);
/* Stop the scheduler after the requests already submitted have completed.  Requests
 * still queued whose tables can no longer fit (the arena is held by results that were
 * not released) end with SIEVE_EBUSY instead, so this call always returns. */
void sieve_server_destroy(sieve_server *srv);

#ifdef __cplusplus
}
#endif

#endif /* GBSIEVE_H */
