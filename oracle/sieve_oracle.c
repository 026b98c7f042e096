/*
 * CPU oracle for the odd-only segmented sieve of Eratosthenes
 * (Jarai & Vatai, "Cache optimized linear sieve", 2011).
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product library links, loads or
 * calls this file; only the tests, the smoke check and the CPU-baseline leg of
 * the benchmark do.  It shares no code, table or header with the CUDA path.
 *
 * What it computes (Definition "Sieve table, Segments", Sec. 1.3): for
 * 0 <= j < n*2^l the bit S_j stands for the odd number 2(f*2^l + j) + 1 and is 1
 * exactly when that number is composite.  The paper's input parameters (Sec.
 * 1.2.1) give the interval u = f*2^(l+1) + 1 .. v = (f+n)*2^(l+1).
 *
 * Everything is exact integer arithmetic (64-bit, with unsigned __int128 for
 * products and remainders), written to be checked by eye, not to be fast:
 *   - base primes: the plain (unsegmented) odd-only sieve of Eratosthenes
 *     (Sec. 1.1, Sec. 1.4 "base" P = primes 2 < p <= sqrt(v));
 *   - the table: segment by segment (Sec. 1.3, Sec. 2.4), every base prime
 *     marks its odd multiples in the segment starting at max(p^2, first odd
 *     multiple in the segment) (Sec. 1.4: sieving with p can start at p^2);
 *     the first multiple comes from the congruence 2J+1 = 0 (mod p), i.e.
 *     J = (p-1)/2 (mod p), not from the parity split of Lemma lem:q, so that
 *     the Lemma can be tested against it;
 *   - deterministic Miller-Rabin and trial division, used only to pin the
 *     sieve in tests.
 * Bit packing: bit j of a table lives in word j/32 at bit position j%32
 * (least significant bit first).
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#include <pthread.h>

typedef unsigned __int128 u128;

#define ORACLE_OK 0
#define ORACLE_EINVAL 1
#define ORACLE_ERANGE 2
#define ORACLE_ENOMEM 3

/* floor(sqrt(x)) exactly, by integer Newton iteration from above, then a
 * final check r^2 <= x < (r+1)^2 in 128-bit arithmetic (the bound sqrt(v) of
 * Sec. 1.4 read as isqrt(v-1), the largest represented number). */
uint64_t oracle_isqrt(uint64_t x)
{
    if (x < 2) return x;
    int bits = 64 - __builtin_clzll(x);
    uint64_t r = (uint64_t)1 << ((bits + 1) / 2); /* r*r > x */
    for (;;) {
        uint64_t nr = (r + x / r) / 2;
        if (nr >= r) break;
        r = nr;
    }
    while ((u128)r * r > x) r--;
    while ((u128)(r + 1) * (r + 1) <= x) r++;
    return r;
}

/* The base (Sec. 1.4, Definition "base"): all odd primes p with 3 <= p <= limit,
 * ascending, by the plain sieve of Eratosthenes over the odd numbers (Sec. 1.1,
 * even numbers not represented, Sec. 1.2).  Index i stands for 2i+1.
 * If out is NULL only the count is returned.  Returns the number of primes, or
 * (uint64_t)-1 when memory runs out. */
uint64_t oracle_base_primes(uint64_t limit, uint32_t *out, uint64_t out_cap)
{
    if (limit < 3) return 0;
    if (limit > 0xFFFFFFFFull) limit = 0xFFFFFFFFull; /* primes stay 32-bit (Sec. 5) */
    uint64_t top = (limit - 1) / 2;                   /* largest index, 2*top+1 <= limit */
    uint8_t *comp = (uint8_t *)calloc(top + 1, 1);
    if (!comp) return (uint64_t)-1;
    for (uint64_t i = 1; ; i++) {
        uint64_t p = 2 * i + 1;
        if (p * p > limit) break;
        if (comp[i]) continue;
        for (uint64_t j = (p * p - 1) / 2; j <= top; j += p) comp[j] = 1;
    }
    uint64_t cnt = 0;
    for (uint64_t i = 1; i <= top; i++) {
        if (comp[i]) continue;
        if (out) {
            if (cnt >= out_cap) { free(comp); return (uint64_t)-1; }
            out[cnt] = (uint32_t)(2 * i + 1);
        }
        cnt++;
    }
    free(comp);
    return cnt;
}

/* One segment of the table (Sec. 1.3): the bits for absolute indices
 * J_start .. J_start+len-1 (number 2J+1), as one byte per bit in seg[]. */
static void sieve_one_segment(uint64_t J_start, uint64_t len,
                              const uint32_t *base, uint64_t nbase, uint8_t *seg)
{
    memset(seg, 0, len);
    /* largest number represented in this segment */
    u128 m_last = 2 * ((u128)J_start + len - 1) + 1;
    for (uint64_t i = 0; i < nbase; i++) {
        uint64_t p = base[i];
        if ((u128)p * p > m_last) break; /* ascending base: no later prime marks here */
        /* first J >= J_start with p | 2J+1, i.e. J = (p-1)/2 (mod p) */
        uint64_t r = J_start % p;
        uint64_t step = ((p - 1) / 2 + p - r) % p;
        u128 J = (u128)J_start + step;
        /* start at p^2 (Sec. 1.4): the index of p^2 is (p^2-1)/2 */
        u128 Jsq = ((u128)p * p - 1) / 2;
        if (J < Jsq) J = Jsq;
        for (u128 k = J - J_start; k < len; k += p) seg[(uint64_t)k] = 1;
    }
}

/* pack bytes (one per bit) into LSB-first 32-bit words; len % 32 == 0 */
static void pack_bits(const uint8_t *seg, uint64_t len, uint32_t *words)
{
    for (uint64_t w = 0; w < len / 32; w++) {
        uint32_t x = 0;
        for (int b = 0; b < 32; b++)
            if (seg[32 * w + b]) x |= (uint32_t)1 << b;
        words[w] = x;
    }
}

typedef struct {
    uint64_t j0, nbits, seg_bits;
    const uint32_t *base;
    uint64_t nbase;
    uint32_t *out;
    uint64_t nseg;
    int tid, nthreads;
    int err;
} seg_job;

static void *seg_worker(void *arg)
{
    seg_job *jb = (seg_job *)arg;
    uint8_t *seg = (uint8_t *)malloc(jb->seg_bits);
    if (!seg) { jb->err = ORACLE_ENOMEM; return NULL; }
    /* static, interleaved assignment of segments to threads */
    for (uint64_t t = (uint64_t)jb->tid; t < jb->nseg; t += (uint64_t)jb->nthreads) {
        uint64_t off = t * jb->seg_bits;
        uint64_t len = jb->nbits - off < jb->seg_bits ? jb->nbits - off : jb->seg_bits;
        sieve_one_segment(jb->j0 + off, len, jb->base, jb->nbase, seg);
        pack_bits(seg, len, jb->out + off / 32);
    }
    free(seg);
    return NULL;
}

/* The table for absolute bit indices j0 .. j0+nbits-1 processed in segments of
 * seg_bits bits (Sec. 1.3 with 2^l = seg_bits, Sec. 2.4: segment after segment;
 * the segments are independent, so they may be handed to several threads).
 * base must hold every odd prime <= base_limit ascending, and base_limit must be
 * >= isqrt of the largest represented number.  j0, nbits, seg_bits multiples of
 * 32.  out receives nbits/32 words. */
int oracle_sieve_range(uint64_t j0, uint64_t nbits, uint64_t seg_bits,
                       const uint32_t *base, uint64_t nbase, uint64_t base_limit,
                       uint32_t *out, int nthreads)
{
    if (nbits == 0) return ORACLE_OK;
    if (j0 % 32 || nbits % 32 || seg_bits == 0 || seg_bits % 32) return ORACLE_EINVAL;
    if (j0 + nbits < j0 || j0 + nbits > ((uint64_t)1 << 63)) return ORACLE_ERANGE;
    uint64_t m_last = 2 * (j0 + nbits - 1) + 1;
    if (oracle_isqrt(m_last) > base_limit) return ORACLE_ERANGE;
    if (nthreads < 1) nthreads = 1;
    uint64_t nseg = (nbits + seg_bits - 1) / seg_bits;
    if ((uint64_t)nthreads > nseg) nthreads = (int)nseg;
    seg_job *jobs = (seg_job *)calloc((size_t)nthreads, sizeof(seg_job));
    pthread_t *th = (pthread_t *)calloc((size_t)nthreads, sizeof(pthread_t));
    if (!jobs || !th) { free(jobs); free(th); return ORACLE_ENOMEM; }
    for (int i = 0; i < nthreads; i++) {
        seg_job j = {j0, nbits, seg_bits, base, nbase, out, nseg, i, nthreads, 0};
        jobs[i] = j;
    }
    for (int i = 1; i < nthreads; i++) pthread_create(&th[i], NULL, seg_worker, &jobs[i]);
    seg_worker(&jobs[0]);
    for (int i = 1; i < nthreads; i++) pthread_join(th[i], NULL);
    int err = ORACLE_OK;
    for (int i = 0; i < nthreads; i++) if (jobs[i].err) err = jobs[i].err;
    free(jobs);
    free(th);
    return err;
}

/* The paper's parameterisation (Sec. 1.2.1): l, f, n -> table of n*2^l bits for
 * the numbers u = f*2^(l+1)+1 .. v = (f+n)*2^(l+1); segments of 2^l bits. */
int oracle_sieve(uint32_t l, uint64_t f, uint64_t n,
                 const uint32_t *base, uint64_t nbase, uint64_t base_limit,
                 uint32_t *out, int nthreads)
{
    if (l < 5 || l > 40 || n == 0) return ORACLE_EINVAL;
    u128 jend = ((u128)f + n) << l;
    if (jend > ((u128)1 << 63)) return ORACLE_ERANGE;
    return oracle_sieve_range(f << l, n << l, (uint64_t)1 << l,
                              base, nbase, base_limit, out, nthreads);
}

/* Lemma lem:q (Sec. 2.1), in the paper's own form: r = f*2^(l+1) mod p, then
 * q = (p-r-1)/2 when r is even and q = (2p-r-1)/2 when r is odd. */
uint64_t oracle_lemma_q(uint64_t p, uint64_t f, uint32_t l)
{
    u128 x = (u128)f << (l + 1);
    uint64_t r = (uint64_t)(x % p);
    return (r % 2 == 0) ? (p - r - 1) / 2 : (2 * p - r - 1) / 2;
}

/* Reading of the midpoint input (Sec. 1.2.1, footnote): with the midpoint
 * M = mant * 10^exp10, choose f so that the interval's midpoint
 * (f + n/2) * 2^(l+1) is M rounded down to the segment grid:
 * f = max(0, floor(M / 2^(l+1)) - floor(n/2)). */
int oracle_f_from_midpoint(uint32_t l, uint64_t n, uint64_t mant, uint32_t exp10, uint64_t *f_out)
{
    if (l < 5 || l > 40) return ORACLE_EINVAL;
    u128 M = mant;
    for (uint32_t i = 0; i < exp10; i++) {
        M *= 10;
        if (M >> 64) return ORACLE_ERANGE;
    }
    u128 q = M >> (l + 1);
    u128 h = n / 2;
    *f_out = q > h ? (uint64_t)(q - h) : 0;
    return ORACLE_OK;
}

/* number of 1 bits (composites) in a packed table */
uint64_t oracle_popcount(const uint32_t *words, uint64_t nwords)
{
    uint64_t c = 0;
    for (uint64_t i = 0; i < nwords; i++) c += (uint64_t)__builtin_popcount(words[i]);
    return c;
}

/* ---- pins: primality by other means --------------------------------------*/

/* trial division: 1 iff m is composite (m > 1 and not prime) */
int oracle_is_composite_trial(uint64_t m)
{
    if (m < 4) return 0;
    if (m % 2 == 0) return 1;
    for (uint64_t d = 3; (u128)d * d <= m; d += 2)
        if (m % d == 0) return 1;
    return 0;
}

static uint64_t mulmod(uint64_t a, uint64_t b, uint64_t m) { return (uint64_t)(((u128)a * b) % m); }

static uint64_t powmod(uint64_t a, uint64_t e, uint64_t m)
{
    uint64_t r = 1 % m;
    a %= m;
    while (e) {
        if (e & 1) r = mulmod(r, a, m);
        a = mulmod(a, a, m);
        e >>= 1;
    }
    return r;
}

/* Deterministic Miller-Rabin for 64-bit m: the twelve prime bases 2..37 decide
 * every m < 3.18e23 (Sorenson & Webster, Math. Comp. 86 (2017)). */
int oracle_is_prime_mr(uint64_t m)
{
    static const uint64_t bases[12] = {2, 3, 5, 7, 11, 13, 17, 19, 23, 29, 31, 37};
    if (m < 2) return 0;
    for (int i = 0; i < 12; i++) {
        if (m == bases[i]) return 1;
        if (m % bases[i] == 0) return 0;
    }
    uint64_t d = m - 1;
    int s = 0;
    while (d % 2 == 0) { d /= 2; s++; }
    for (int i = 0; i < 12; i++) {
        uint64_t x = powmod(bases[i], d, m);
        if (x == 1 || x == m - 1) continue;
        int witness = 1;
        for (int k = 1; k < s; k++) {
            x = mulmod(x, x, m);
            if (x == m - 1) { witness = 0; break; }
        }
        if (witness) return 0;
    }
    return 1;
}

/* bit j of a table as 0/1 */
int oracle_get_bit(const uint32_t *words, uint64_t j)
{
    return (int)((words[j / 32] >> (j % 32)) & 1u);
}

/* Consumers of a finished table (Sec. 5: the table is made to be used, e.g. for
 * prime counts and the Goldbach search): per segment of 2^l bits, the primes and
 * the twin pairs.  Bit j (0 <= j < nbits) of `words` stands for m = 2(J0 + j) + 1;
 * m is a prime when the bit is 0 and m != 1 (the table's 0 bits are exactly the
 * primes and the number 1).  A twin pair is (m, m + 2) with both prime; m + 2 is
 * bit j + 1, so the pair is counted only when j + 1 < nbits, in the segment j >> l
 * of its lower member.  Plain loop over bits; primes[] and twins[] hold
 * ceil(nbits / 2^l) entries and are overwritten. */
int oracle_segment_counts(const uint32_t *words, uint64_t J0, uint64_t nbits, uint32_t l,
                          uint64_t *primes, uint64_t *twins)
{
    if (l > 62 || (nbits && !words)) return ORACLE_EINVAL;
    const uint64_t nseg = (nbits + ((uint64_t)1 << l) - 1) >> l;
    for (uint64_t t = 0; t < nseg; ++t) primes[t] = twins[t] = 0;
    int prev_prime = 0; /* bit j - 1 is a prime */
    for (uint64_t j = 0; j < nbits; ++j) {
        const int is_prime = oracle_get_bit(words, j) == 0 && J0 + j != 0;
        if (is_prime) primes[j >> l]++;
        if (is_prime && prev_prime) twins[(j - 1) >> l]++;
        prev_prime = is_prime;
    }
    return ORACLE_OK;
}

/* Goldbach search (Sec. 5: the sieve is made for verifying the Goldbach conjecture).
 * For the even numbers N = n_lo + 2i, 0 <= i < count: min_p[i] = the smallest odd
 * prime p among primes[0..nprimes) (ascending odd primes) with p <= p_max such that
 * N - p is prime, decided by deterministic Miller-Rabin (oracle_is_prime_mr), not by a
 * sieve; 0 when there is none.  Plain double loop. */
int oracle_goldbach_min_p(uint64_t n_lo, uint64_t count, const uint32_t *primes, uint64_t nprimes,
                          uint32_t p_max, uint32_t *min_p)
{
    if ((n_lo & 1) || (count && !min_p) || (nprimes && !primes)) return ORACLE_EINVAL;
    for (uint64_t i = 0; i < count; ++i) {
        const uint64_t N = n_lo + 2 * i;
        min_p[i] = 0;
        for (uint64_t k = 0; k < nprimes && primes[k] <= p_max; ++k) {
            const uint64_t p = primes[k];
            if (p + 3 > N) break; /* N - p >= 3: the smallest odd prime */
            if (oracle_is_prime_mr(N - p)) {
                min_p[i] = (uint32_t)p;
                break;
            }
        }
    }
    return ORACLE_OK;
}
