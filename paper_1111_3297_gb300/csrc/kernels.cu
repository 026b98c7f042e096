// Device kernels of the GB300 sieve (sm_103a).
//
//   k_tile       one on-chip segment ("tile", Sec. 1.3 segments) per CTA, persistent
//                grid: pre-sieve by pattern copy (Sec. 3.1), medium primes striding
//                through shared memory with the mod-15 wheel (Sec. 2.1, Sec. 3.2.1),
//                drain of the tile's large-prime bucket (Sec. 2.2-2.3), coalesced
//                128-bit store and popcount.
//   k_scatter_run, k_scatter   large primes (stride beyond the tile) into per-tile
//                buckets in HBM: hits staged per warp in shared memory, counting-sorted
//                by tile, appended with one atomic reservation per (tile, flush).  One
//                interval: each prime's next hit and wheel position live in one state
//                word through the whole interval.  Several requests: first hit per
//                (prime, request unit) by Barrett reduction (Lemma lem:q, Sec. 1.4).
//   k_bootstrap, k_compact_*, k_barrett   the base of Sec. 1.4 built on the device.
//   k_popcount   composite count of a table.
//   k_probe_smem shared-memory atomic-OR rate (roofline denominator).
#include "sieve_internal.cuh"

namespace gbs {

__constant__ uint32_t c_cum[8] = {pack_cum(0), pack_cum(1), pack_cum(2), pack_cum(3),
                                  pack_cum(4), pack_cum(5), pack_cum(6), pack_cum(7)};

// bit (q-1)/2 set for every odd prime q <= 127: a pre-sieve pattern marks q*1 = q
// itself, which is prime, so those bits are cleared again where they occur
constexpr uint64_t small_prime_bits()
{
    uint64_t x = 0;
    for (int q = 3; q <= 127; q += 2) {
        bool pr = true;
        for (int d = 3; d * d <= q; d += 2)
            if (q % d == 0) pr = false;
        if (pr) x |= 1ull << ((q - 1) / 2);
    }
    return x;
}
constexpr uint64_t kSmallPrimeBits = small_prime_bits();

__device__ __forceinline__ uint32_t lanemask_lt()
{
    uint32_t m;
    asm("mov.u32 %0, %%lanemask_lt;" : "=r"(m));
    return m;
}

// block-wide exclusive scan of one value per thread (T threads); returns the
// exclusive prefix, total in *tot
template <int T>
__device__ __forceinline__ uint32_t block_excl_scan(uint32_t v, uint32_t *s_warp, uint32_t *tot)
{
    const uint32_t lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    uint32_t incl = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const uint32_t y = __shfl_up_sync(0xffffffffu, incl, o);
        if (lane >= (uint32_t)o) incl += y;
    }
    if (lane == 31) s_warp[warp] = incl;
    __syncthreads();
    if (warp == 0) {
        uint32_t w = lane < T / 32 ? s_warp[lane] : 0;
        uint32_t wi = w;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const uint32_t y = __shfl_up_sync(0xffffffffu, wi, o);
            if (lane >= (uint32_t)o) wi += y;
        }
        if (lane < T / 32) s_warp[lane] = wi - w;
        if (lane == T / 32 - 1) s_warp[32] = wi;
    }
    __syncthreads();
    const uint32_t r = s_warp[warp] + incl - v;
    *tot = s_warp[32];
    __syncthreads();
    return r;
}

// ---------------------------------------------------------------------------
// tile kernel
// ---------------------------------------------------------------------------

// One pre-sieve pass over the tile's words: OR of the patterns of groups
// [G0, G0 + NG) (Sec. 3.1).  Thread tid takes words tid, tid + T, ...; the
// pattern window of group g for word w starts at rho = (J + 32 w) mod P_g.  The
// first pass (G0 = 0) writes the words, a later one ORs into them; the last pass
// also clears the bits of the small primes themselves (q = q * 1 is prime).
template <int T, int G0, int NG>
__device__ __forceinline__ void presieve_pass(uint32_t *sm, const TileArgs &a, const uint32_t *s_rho0,
                                              uint32_t nwords, bool last, uint64_t J)
{
    const uint32_t tid = threadIdx.x;
    uint32_t rho[NG];
#pragma unroll
    for (int k = 0; k < NG; ++k) {
        // rho = (rho0 + 32 tid) mod P: the quotient estimated in float, corrected exactly
        const uint32_t P = a.ps.modulus[G0 + k], x = 32u * tid;
        const uint32_t q = __float2uint_rz(__uint2float_rn(x) * a.ps.inv[G0 + k]);
        int32_t r = (int32_t)(x - q * P);
        if (r < 0) r += (int32_t)P;
        if (r >= (int32_t)P) r -= (int32_t)P;
        const uint32_t r2 = s_rho0[G0 + k] + (uint32_t)r;
        rho[k] = r2 >= P ? r2 - P : r2;
    }
    for (uint32_t w = tid; w < nwords; w += T) {
        uint32_t mask = G0 ? sm[w] : 0u;
#pragma unroll
        for (int k = 0; k < NG; ++k) {
            const uint32_t r = rho[k];
            mask |= (uint32_t)(__ldg(a.pat + a.ps.word_off[G0 + k] + (r >> 5)) >> (r & 31));
            const uint32_t nr = r + a.ps.inc[G0 + k];
            rho[k] = nr >= a.ps.modulus[G0 + k] ? nr - a.ps.modulus[G0 + k] : nr;
        }
        if (last) {
            const uint64_t Jw = J + 32ull * w;
            if (Jw < 64) mask &= ~(uint32_t)(kSmallPrimeBits >> Jw);
        }
        sm[w] = mask;
    }
}
// Count mode of the finished tile in shared memory (Sec. 5: the table consumed where it
// is made).  A zero bit j is a prime 2(J+j)+1, except the number 1; a twin pair is two
// adjacent zero bits (the odd numbers m and m+2).  The host guarantees 2^seg_l >= 4096
// and tiles of whole 4096-bit chunks starting 4096-aligned relative to seg_j0, so the
// 32 uint4 words a warp reads in one trip lie in one segment.  The pair formed by the
// tile's last bit and the next tile's first bit is left to k_seg_edges.
template <int T>
__device__ __forceinline__ void tile_counts(const uint32_t *sm, const TileArgs &a, const TileDesc &d,
                                            uint32_t t, uint32_t nwords, uint32_t *s_red)
{
    const uint32_t tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const uint32_t n4 = nwords >> 2;  // a multiple of 32
    const uint4 *s4 = reinterpret_cast<const uint4 *>(sm);
    const bool per_chunk = a.seg_l < a.tile_log2;  // several segments per tile
    uint32_t tp = 0, tt = 0;
    for (uint32_t i = tid; i < n4; i += T) {
        const uint4 v = s4[i];
        const uint32_t z0 = ~v.x, z1 = ~v.y, z2 = ~v.z, z3 = ~v.w;
        const uint32_t z4 = 4 * i + 4 < nwords ? ~sm[4 * i + 4] : 0u;  // past the tile: left to k_seg_edges
        uint32_t pc = __popc(z0) + __popc(z1) + __popc(z2) + __popc(z3);
        uint32_t tc = __popc(z0 & ((z0 >> 1) | (z1 << 31))) + __popc(z1 & ((z1 >> 1) | (z2 << 31))) +
                      __popc(z2 & ((z2 >> 1) | (z3 << 31))) + __popc(z3 & ((z3 >> 1) | (z4 << 31)));
        if (i == 0 && d.J == 0) {
            pc -= z0 & 1u;          // the number 1 is not a prime
            tc -= z0 & (z0 >> 1) & 1u;  // nor is (1, 3) a twin pair
        }
        if (per_chunk) {
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) {
                pc += __shfl_xor_sync(0xffffffffu, pc, o);
                tc += __shfl_xor_sync(0xffffffffu, tc, o);
            }
            if (lane == 0) {
                const uint64_t seg = (d.J + 128ull * (i - lane) - a.seg_j0) >> a.seg_l;
                atomicAdd(&a.seg_primes[seg], (unsigned long long)pc);
                if (a.seg_twins) atomicAdd(&a.seg_twins[seg], (unsigned long long)tc);
            }
        } else {
            tp += pc;
            tt += tc;
        }
    }
    if (!per_chunk) {
        // the tile lies in one segment: one pair of atomics per tile
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            tp += __shfl_xor_sync(0xffffffffu, tp, o);
            tt += __shfl_xor_sync(0xffffffffu, tt, o);
        }
        if (lane == 0) {
            s_red[warp] = tp;
            s_red[T / 32 + warp] = tt;
        }
        __syncthreads();
        if (warp == 0) {
            uint32_t x = lane < T / 32 ? s_red[lane] : 0, y = lane < T / 32 ? s_red[T / 32 + lane] : 0;
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) {
                x += __shfl_xor_sync(0xffffffffu, x, o);
                y += __shfl_xor_sync(0xffffffffu, y, o);
            }
            if (lane == 0) {
                const uint64_t seg = (d.J - a.seg_j0) >> a.seg_l;
                atomicAdd(&a.seg_primes[seg], (unsigned long long)x);
                if (a.seg_twins) atomicAdd(&a.seg_twins[seg], (unsigned long long)y);
            }
        }
    }
    if (tid == 0) {
        const uint32_t first = (d.J == 0) ? 0u : (~sm[0] & 1u);
        a.edge[t] = (uint8_t)(first | (((~sm[nwords - 1]) >> 31) << 1));
    }
    __syncthreads();
}

// thread-block cluster helpers (PTX: %cluster_ctarank, %cluster_nctarank, barrier.cluster)
__device__ __forceinline__ uint32_t cluster_rank()
{
    uint32_t r;
    asm volatile("mov.u32 %0, %%cluster_ctarank;" : "=r"(r));
    return r;
}
__device__ __forceinline__ uint32_t cluster_size()
{
    uint32_t r;
    asm volatile("mov.u32 %0, %%cluster_nctarank;" : "=r"(r));
    return r;
}
__device__ __forceinline__ void cluster_barrier()
{
    asm volatile("barrier.cluster.arrive.release.aligned;\n\tbarrier.cluster.wait.acquire.aligned;" ::: "memory");
}

// Pre-sieve of the words [0, nwords) of a tile (or cluster slice) starting at index J.
template <int T>
__device__ __forceinline__ void presieve_tile(uint32_t *sm, const TileArgs &a, uint32_t *s_rho0, uint64_t J,
                                              uint32_t nwords)
{
    const uint32_t tid = threadIdx.x;
    const uint32_t ng = a.ps.ngroups;
    // ---- pre-sieve: OR of the small-prime patterns (Sec. 3.1) ----
    // Passes of at most 7 groups (fewer live residues per thread), each compiled
    // for its exact groups; the second pass ORs into the words the first wrote.
    if (tid < ng) s_rho0[tid] = mod_barrett(J, a.ps.modulus[tid], a.ps.barrett[tid]);
    __syncthreads();
    switch (ng < 7 ? ng : 7) {
    case 1: presieve_pass<T, 0, 1>(sm, a, s_rho0, nwords, ng <= 7, J); break;
    case 2: presieve_pass<T, 0, 2>(sm, a, s_rho0, nwords, ng <= 7, J); break;
    case 3: presieve_pass<T, 0, 3>(sm, a, s_rho0, nwords, ng <= 7, J); break;
    case 4: presieve_pass<T, 0, 4>(sm, a, s_rho0, nwords, ng <= 7, J); break;
    case 5: presieve_pass<T, 0, 5>(sm, a, s_rho0, nwords, ng <= 7, J); break;
    case 6: presieve_pass<T, 0, 6>(sm, a, s_rho0, nwords, ng <= 7, J); break;
    default: presieve_pass<T, 0, 7>(sm, a, s_rho0, nwords, ng <= 7, J); break;
    }
    switch (ng > 7 ? ng - 7 : 0) {
    case 0: break;
    case 1: presieve_pass<T, 7, 1>(sm, a, s_rho0, nwords, true, J); break;
    case 2: presieve_pass<T, 7, 2>(sm, a, s_rho0, nwords, true, J); break;
    case 3: presieve_pass<T, 7, 3>(sm, a, s_rho0, nwords, true, J); break;
    case 4: presieve_pass<T, 7, 4>(sm, a, s_rho0, nwords, true, J); break;
    case 5: presieve_pass<T, 7, 5>(sm, a, s_rho0, nwords, true, J); break;
    default: presieve_pass<T, 7, 6>(sm, a, s_rho0, nwords, true, J); break;
    }
    __syncthreads();
}

// Medium primes with many hits per tile, struck by the whole CTA and by one warp per
// prime, over the len bits of a tile (or cluster slice) starting at index J.
template <int T>
__device__ __forceinline__ void strike_small_medium(uint32_t *sm, const TileArgs &a, uint64_t J, uint32_t len,
                                                    uint32_t med_hi)
{
    const uint32_t lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    // ---- medium primes (Sec. 2.1, Sec. 3.2), wheel of Sec. 3.2.1 ----
    // A lane strikes the (lane%8)-th admissible multiple of wheel period lane/8
    // (a period is 15 multiples of p, 8 of them admissible), so a warp covers 4
    // periods = 60 multiples of p per step.
    const uint32_t js15 = (uint32_t)(J % 15u);
    const uint32_t cum_shift = 4u * (lane & 7), lane_base = 15u * (lane >> 3);
    {
        // smallest primes: every warp takes every prime and strikes every NW-th
        // step of it (warp w: steps w, w + NW, ...), so the work of one prime is
        // spread over the whole CTA and a warp's start is one multiply-add
        constexpr uint32_t NW = T / 32;
        const uint32_t blk_end = min(a.blk_hi, med_hi);
        for (uint32_t b = a.med_lo; b < blk_end; b += 32) {
            const uint32_t idx = b + lane;
            uint32_t p = 0, h = len, s = 0;
            if (idx < blk_end) {
                p = a.primes[idx];
                const uint64_t hh = first_hit(J, js15, p, a.barrett[idx], s);
                h = hh < len ? (uint32_t)hh : len;
            }
            for (int j = 0; j < 32; ++j) {
                const uint32_t hj = __shfl_sync(0xffffffffu, h, j);
                const uint32_t pj = __shfl_sync(0xffffffffu, p, j);
                const uint32_t sj = __shfl_sync(0xffffffffu, s, j);
                if (hj >= len) continue;
                // the host gives this phase primes with 4 * NW steps <= the tile, so
                // pos stays below len + NW * step < 2^21
                const uint32_t step = 60u * pj, stride = NW * step;
                uint32_t pos = hj + (lane_base + ((c_cum[sj] >> cum_shift) & 15u)) * pj + warp * step;
                while (pos < len) {
                    atomicOr(&sm[pos >> 5], 1u << (pos & 31));
                    pos += stride;
                }
            }
        }
    }
    {
        // one prime per warp at a time; a warp's 32 primes are dealt round-robin
        // from the whole range so that the warps' loads even out
        constexpr uint32_t NW = T / 32;
        const uint32_t lo = max(a.med_lo, a.blk_hi);
        const uint32_t coop_end = min(a.coop_hi, med_hi);
        for (uint32_t b = lo; b < coop_end; b += 32 * NW) {
            const uint32_t idx = b + lane * NW + warp;
            uint32_t p = 0, h = len, s = 0;
            if (idx < coop_end) {
                p = a.primes[idx];
                const uint64_t hh = first_hit(J, js15, p, a.barrett[idx], s);
                h = hh < len ? (uint32_t)hh : len;
            }
            for (int j = 0; j < 32; ++j) {
                const uint32_t hj = __shfl_sync(0xffffffffu, h, j);
                const uint32_t pj = __shfl_sync(0xffffffffu, p, j);
                const uint32_t sj = __shfl_sync(0xffffffffu, s, j);
                if (hj >= len) continue;
                uint32_t pos = hj + (lane_base + ((c_cum[sj] >> cum_shift) & 15u)) * pj;
                const uint32_t step = 60u * pj;
                while (pos < len) {
                    atomicOr(&sm[pos >> 5], 1u << (pos & 31));
                    pos += step;
                }
            }
        }
    }
}

template <int T>
__global__ void __launch_bounds__(T, 2048 / T) k_tile(TileArgs a)
{
    extern __shared__ __align__(16) uint32_t sm[];
    __shared__ uint32_t s_tile;
    __shared__ uint32_t s_rho0[kMaxPresieveGroups];
    __shared__ uint32_t s_red[2 * (T / 32)];
    const uint32_t tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const uint32_t ng = a.ps.ngroups;

    const uint32_t run_lo = a.run ? blockIdx.x * a.run : 0u;
    const uint32_t run_hi = a.run ? min(a.ntiles, run_lo + a.run) : 0u;
    for (uint32_t it = 0;; ++it) {
        if (a.run) {
            if (run_lo + it >= run_hi) break;
            if (tid == 0) s_tile = run_lo + it;
        } else if (tid == 0) {
            s_tile = atomicAdd(a.work, 1u);
        }
        __syncthreads();
        const uint32_t t = s_tile;
        if (t >= a.ntiles) break;
        const TileDesc d = a.tiles[t];
        const uint32_t len = d.len, nwords = len >> 5;
        const bool carried = a.run && it > 0;  // the previous tile of this CTA ends where d starts

        presieve_tile<T>(sm, a, s_rho0, d.J, nwords);

        const uint32_t js15 = (uint32_t)(d.J % 15u);
        strike_small_medium<T>(sm, a, d.J, len, d.med_hi);
        {
            // one prime per thread, the next prime's loads issued ahead; in a run of
            // tiles the next hit carries over (relative to the next tile's start)
            const uint32_t end = d.med_hi;
            const uint32_t lo = max(max(a.med_lo, a.blk_hi), a.coop_hi);
            // carried state: next hit offset (29 bits; all ones = beyond the run) and
            // wheel state (3 bits)
            uint32_t *ch = a.carry_h + (size_t)blockIdx.x * a.carry_stride - lo;
            uint32_t idx = lo + tid;
            uint32_t pn = 0, cn = 0;
            uint64_t mn = 0;
            if (idx < end) {
                pn = a.primes[idx];
                if (carried)
                    cn = ch[idx];
                else
                    mn = a.barrett[idx];
            }
            while (idx < end) {
                const uint32_t p = pn;
                const uint64_t m = mn;
                const uint32_t cc = cn;
                const uint32_t nidx = idx + T;
                if (nidx < end) {
                    pn = a.primes[nidx];
                    if (carried)
                        cn = ch[nidx];
                    else
                        mn = a.barrett[nidx];
                }
                // next hit offset in the tile, or kNone when at or beyond len + 2^29 - 1
                // (medium primes < 2^28: every offset below fits 32 bits)
                constexpr uint32_t kNone = 0xFFFFFFFFu;
                uint32_t s = cc >> 29;
                uint32_t h = (cc & 0x1FFFFFFFu) == 0x1FFFFFFFu ? kNone : (cc & 0x1FFFFFFFu);
                if (!carried) {
                    const uint64_t f = first_hit(d.J, js15, p, m, s);
                    h = f < (uint64_t)len + 0x1FFFFFFFu ? (uint32_t)f : kNone;
                }
                if (h < len) {
                    // gaps of the mod-15 wheel from state s on, 2 bits each: the packed
                    // cycle doubled to 32 bits, so a rotate by 2 is one wheel step
                    uint32_t gq = __funnelshift_r(kGapPacked * 0x10001u, kGapPacked * 0x10001u, 2 * s), k = 0;
                    for (;;) {
                        atomicOr(&sm[h >> 5], 1u << (h & 31));
                        h += (gq & 3u) * p;  // medium primes < 2^28: no overflow
                        gq = __funnelshift_r(gq, gq, 2);
                        ++k;
                        if (h >= len) break;
                    }
                    s = (s + k) & 7;
                }
                if (a.run) {
                    // next hit relative to the next tile; all ones (kept as is) when it
                    // lies beyond the run, which spans less than 2^29 - 1 bits
                    const uint32_t off = h >= len + 0x1FFFFFFFu ? 0x1FFFFFFFu : h - len;
                    ch[idx] = (s << 29) | off;
                }
                idx = nidx;
            }
        }

        // ---- drain the tile's large-prime bucket (Sec. 2.2-2.3) ----
        if (d.bkt_cap) {
            const uint32_t cnt = min(a.bkt_cnt[t], d.bkt_cap);
            const uint32_t *e = a.bkt + d.bkt_off;
            const uint32_t n4 = cnt >> 2;
            const uint4 *e4 = reinterpret_cast<const uint4 *>(e);
#pragma unroll 4  // several 16-byte loads in flight per thread
            for (uint32_t i = tid; i < n4; i += T) {
                const uint4 v = __ldcs(e4 + i);
                atomicOr(&sm[v.x >> 5], 1u << (v.x & 31));
                atomicOr(&sm[v.y >> 5], 1u << (v.y & 31));
                atomicOr(&sm[v.z >> 5], 1u << (v.z & 31));
                atomicOr(&sm[v.w >> 5], 1u << (v.w & 31));
            }
            for (uint32_t i = 4 * n4 + tid; i < cnt; i += T) {
                const uint32_t v = __ldcs(e + i);
                atomicOr(&sm[v >> 5], 1u << (v & 31));
            }
            const uint32_t oc = min(*(volatile const uint32_t *)a.ovf_cnt, a.ovf_cap);
            for (uint32_t i = tid; i < oc; i += T) {
                const unsigned long long x = a.ovf[i];
                if ((uint32_t)(x >> 32) == t) {
                    const uint32_t v = (uint32_t)x;
                    atomicOr(&sm[v >> 5], 1u << (v & 31));
                }
            }
        }
        __syncthreads();

        // ---- count mode: primes and twin pairs per segment, no table written ----
        if (!a.out) {
            tile_counts<T>(sm, a, d, t, nwords, s_red);
            continue;
        }

        // ---- store (128-bit when aligned) and popcount ----
        uint32_t pop = 0;
        uint32_t *out = a.out + d.out_word;
        if (((reinterpret_cast<uintptr_t>(out) & 15) == 0) && ((nwords & 3) == 0)) {
            uint4 *o4 = reinterpret_cast<uint4 *>(out);
            const uint4 *s4 = reinterpret_cast<const uint4 *>(sm);
            for (uint32_t i = tid; i < (nwords >> 2); i += T) {
                const uint4 v = s4[i];
                o4[i] = v;
                pop += __popc(v.x) + __popc(v.y) + __popc(v.z) + __popc(v.w);
            }
        } else {
            for (uint32_t i = tid; i < nwords; i += T) {
                const uint32_t v = sm[i];
                out[i] = v;
                pop += __popc(v);
            }
        }
        if (a.req_counts) {
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) pop += __shfl_xor_sync(0xffffffffu, pop, o);
            if (lane == 0) s_red[warp] = pop;
            __syncthreads();
            if (warp == 0) {
                uint32_t v = lane < T / 32 ? s_red[lane] : 0;
#pragma unroll
                for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
                if (lane == 0) atomicAdd(&a.req_counts[d.req], (unsigned long long)v);
            }
        }
        __syncthreads();
    }
}

// ---------------------------------------------------------------------------
// Cluster tile kernel: one segment of up to C * 2^20 bits held across the shared
// memory of a cluster of C CTAs (Sec. 2.2: a larger segment leaves fewer primes
// large), CTA rank r owning the slice [r * 2^20, (r+1) * 2^20).  Each CTA pre-sieves
// its own slice and strikes the primes with many hits per slice there (the CTA-wide
// and warp-per-prime phases, on its slice alone).  The one-prime-per-thread primes
// and the drained bucket entries cover the whole segment: the C CTAs split them,
// and a strike in another rank's slice is an OR through the cluster window
// (red.shared::cluster).  Every index into a slice is masked to the slice and every
// rank to the cluster, so no access leaves the cluster's shared memory whatever the
// entries hold.
// Cluster barriers: A after the pre-sieve (a slice is written before any rank ORs
// into it), B after the last strike (before the slices are stored).  The next
// tile's remote ORs come after its barrier A, which each CTA reaches only after
// storing its slice.  Cluster c takes the tiles [c * run, (c+1) * run) in order
// (one interval, each tile starting where the previous one ends), so both CTAs of a
// cluster walk the same tiles and reach both barriers the same number of times, on
// every path; a cluster without tiles reaches none.
// ---------------------------------------------------------------------------
template <int C>
__global__ void __launch_bounds__(1024, 1) k_ctile(TileArgs a)
{
    static_assert(C == 2, "two-CTA clusters");
    constexpr int T = 1024;
    constexpr uint32_t SL = 1u << 20;  // bits per slice
    extern __shared__ __align__(16) uint32_t sm[];
    __shared__ uint32_t s_rho0[kMaxPresieveGroups];
    __shared__ uint32_t s_red[T / 32];
    const uint32_t tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const uint32_t rank = cluster_rank() & (C - 1);
    uint32_t cid;
    asm volatile("mov.u32 %0, %%clusterid.x;" : "=r"(cid));
    // cluster-window addresses of the two slices
    const uint32_t local = (uint32_t)__cvta_generic_to_shared(sm);
    uint32_t win0, win1;
    asm volatile("mapa.shared::cluster.u32 %0, %1, 0;" : "=r"(win0) : "r"(local));
    asm volatile("mapa.shared::cluster.u32 %0, %1, 1;" : "=r"(win1) : "r"(local));

    // one bit into slice word (pos & (SL-1)) >> 5 of rank (pos >> 20) & (C-1)
    auto strike = [&](uint32_t pos) {
        const uint32_t owner = (pos >> 20) & (C - 1), loc = pos & (SL - 1);
        const uint32_t bit = 1u << (loc & 31);
        if (owner == rank) {
            atomicOr(&sm[loc >> 5], bit);
        } else {
            const uint32_t addr = (owner ? win1 : win0) + ((loc >> 5) << 2);
            asm volatile("red.relaxed.cluster.shared::cluster.or.b32 [%0], %1;" ::"r"(addr), "r"(bit) : "memory");
        }
    };

    const uint32_t run_lo = cid * a.run;
    const uint32_t run_hi = min(a.ntiles, run_lo + a.run);
    for (uint32_t it = 0; run_lo + it < run_hi; ++it) {
        const uint32_t t = run_lo + it;
        const TileDesc d = a.tiles[t];
        const uint32_t len = d.len;
        const uint64_t Js = d.J + (uint64_t)rank * SL;
        const uint32_t lens = len > rank * SL ? min(SL, len - rank * SL) : 0u;
        const bool carried = it > 0;  // the cluster's previous tile ends where d starts

        presieve_tile<T>(sm, a, s_rho0, Js, lens >> 5);
        cluster_barrier();  // A
        strike_small_medium<T>(sm, a, Js, lens, d.med_hi);

        {
            // one prime per thread over the whole segment, the two CTAs taking alternate
            // blocks of T primes; next hits carried from tile to tile as in k_tile
            const uint32_t js15 = (uint32_t)(d.J % 15u);
            const uint32_t end = d.med_hi;
            const uint32_t lo = max(max(a.med_lo, a.blk_hi), a.coop_hi);
            uint32_t *ch = a.carry_h + (size_t)blockIdx.x * a.carry_stride - lo;
            for (uint32_t idx = lo + rank * T + tid; idx < end; idx += C * T) {
                const uint32_t p = a.primes[idx];
                constexpr uint32_t kNone = 0xFFFFFFFFu;
                uint32_t s = 0, h;
                if (carried) {
                    const uint32_t cc = ch[idx];
                    s = cc >> 29;
                    h = (cc & 0x1FFFFFFFu) == 0x1FFFFFFFu ? kNone : (cc & 0x1FFFFFFFu);
                } else {
                    const uint64_t f = first_hit(d.J, js15, p, a.barrett[idx], s);
                    h = f < (uint64_t)len + 0x1FFFFFFFu ? (uint32_t)f : kNone;
                }
                if (h < len) {
                    uint32_t gq = __funnelshift_r(kGapPacked * 0x10001u, kGapPacked * 0x10001u, 2 * s), k = 0;
                    for (;;) {
                        strike(h);
                        h += (gq & 3u) * p;
                        gq = __funnelshift_r(gq, gq, 2);
                        ++k;
                        if (h >= len) break;
                    }
                    s = (s + k) & 7;
                }
                const uint32_t off = h >= len + 0x1FFFFFFFu ? 0x1FFFFFFFu : h - len;
                ch[idx] = (s << 29) | off;
            }
        }

        // ---- the segment's large-prime bucket, entries split between the CTAs ----
        if (d.bkt_cap) {
            const uint32_t cnt = min(a.bkt_cnt[t], d.bkt_cap);
            const uint32_t *e = a.bkt + d.bkt_off;
            const uint32_t n4 = cnt >> 2;
            const uint4 *e4 = reinterpret_cast<const uint4 *>(e);
#pragma unroll 4
            for (uint32_t i = rank * T + tid; i < n4; i += C * T) {
                const uint4 v = __ldcs(e4 + i);
                strike(v.x);
                strike(v.y);
                strike(v.z);
                strike(v.w);
            }
            for (uint32_t i = 4 * n4 + rank * T + tid; i < cnt; i += C * T) strike(__ldcs(e + i));
            const uint32_t oc = min(*(volatile const uint32_t *)a.ovf_cnt, a.ovf_cap);
            for (uint32_t i = rank * T + tid; i < oc; i += C * T) {
                const unsigned long long x = a.ovf[i];
                if ((uint32_t)(x >> 32) == t) strike((uint32_t)x);
            }
        }
        __syncthreads();    // every warp converged before the cluster barrier
        cluster_barrier();  // B

        // ---- store the own slice (128-bit when aligned) and popcount ----
        const uint32_t nwords = lens >> 5;
        uint32_t pop = 0;
        uint32_t *out = a.out + d.out_word + (size_t)rank * (SL / 32);
        if (((reinterpret_cast<uintptr_t>(out) & 15) == 0) && ((nwords & 3) == 0)) {
            uint4 *o4 = reinterpret_cast<uint4 *>(out);
            const uint4 *s4 = reinterpret_cast<const uint4 *>(sm);
            for (uint32_t i = tid; i < (nwords >> 2); i += T) {
                const uint4 v = s4[i];
                o4[i] = v;
                pop += __popc(v.x) + __popc(v.y) + __popc(v.z) + __popc(v.w);
            }
        } else {
            for (uint32_t i = tid; i < nwords; i += T) {
                const uint32_t v = sm[i];
                out[i] = v;
                pop += __popc(v);
            }
        }
        if (a.req_counts) {
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) pop += __shfl_xor_sync(0xffffffffu, pop, o);
            if (lane == 0) s_red[warp] = pop;
            __syncthreads();
            if (warp == 0) {
                uint32_t v = s_red[lane];
#pragma unroll
                for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
                if (lane == 0 && v) atomicAdd(&a.req_counts[d.req], (unsigned long long)v);
            }
        }
        __syncthreads();  // the slice is stored before the next pre-sieve overwrites it
    }
}

int tile_threads(uint32_t tile_log2) { return tile_log2 >= 17 ? 1024 : (tile_log2 >= 14 ? 512 : 256); }
// a tile (or, beyond 2^20 bits, each CTA's slice of a cluster tile) in shared memory
size_t tile_smem_bytes(uint32_t tile_log2) { return (size_t)1 << ((tile_log2 < 20 ? tile_log2 : 20) - 3); }

// clusters of two 1024-thread CTAs with a 2^20-bit slice each that fit on the GPU at once
int ctile_max_clusters()
{
    static int cached = 0;
    if (cached) return cached;
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeClusterDimension;
    at[0].val.clusterDim.x = 2;
    at[0].val.clusterDim.y = 1;
    at[0].val.clusterDim.z = 1;
    cudaLaunchConfig_t cfg = {};
    cfg.blockDim = dim3(1024);
    cfg.gridDim = dim3(2);
    cfg.dynamicSmemBytes = tile_smem_bytes(20);
    cfg.attrs = at;
    cfg.numAttrs = 1;
    int n = 0;
    if (cudaOccupancyMaxActiveClusters(&n, k_ctile<2>, &cfg) != cudaSuccess || n < 1) {
        cudaGetLastError();
        return 0;
    }
    cached = n;
    return n;
}

// nclusters clusters of two CTAs; a.run tiles per cluster
cudaError_t launch_ctiles(const TileArgs &a, uint32_t nclusters, cudaStream_t st)
{
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeClusterDimension;
    at[0].val.clusterDim.x = 2;
    at[0].val.clusterDim.y = 1;
    at[0].val.clusterDim.z = 1;
    cudaLaunchConfig_t cfg = {};
    cfg.blockDim = dim3(1024);
    cfg.gridDim = dim3(2 * nclusters);
    cfg.dynamicSmemBytes = tile_smem_bytes(20);
    cfg.stream = st;
    cfg.attrs = at;
    cfg.numAttrs = 1;
    const cudaError_t e = cudaLaunchKernelEx(&cfg, k_ctile<2>, a);
    return e != cudaSuccess ? e : cudaGetLastError();
}

template <int T>
static cudaError_t launch_tiles_t(const TileArgs &a, uint32_t grid, cudaStream_t st)
{
    const size_t smem = tile_smem_bytes(a.tile_log2);
    k_tile<T><<<grid, T, smem, st>>>(a);
    return cudaGetLastError();
}

cudaError_t launch_tiles(const TileArgs &a, uint32_t grid, cudaStream_t st)
{
    switch (tile_threads(a.tile_log2)) {
    case 1024: return launch_tiles_t<1024>(a, grid, st);
    case 512: return launch_tiles_t<512>(a, grid, st);
    default: return launch_tiles_t<256>(a, grid, st);
    }
}

int tile_blocks_per_sm(uint32_t tile_log2)
{
    int n = 0;
    const size_t smem = tile_smem_bytes(tile_log2);
    switch (tile_threads(tile_log2)) {
    case 1024:
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k_tile<1024>, 1024, smem);
        break;
    case 512:
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k_tile<512>, 512, smem);
        break;
    default:
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k_tile<256>, 256, smem);
    }
    return n < 1 ? 1 : n;
}

// ---------------------------------------------------------------------------
// scatter kernel: large primes -> per-tile buckets
//
// CTA = one chunk: a run of consecutive large primes (cut on the host so that
// chunks carry similar work), walked through every scatter group of the epoch
// (a group is <= kScatterMaxTiles tiles of one or more requests).  Prime-major: a
// warp takes 32 primes (one per lane, prime and Barrett constant in registers),
// walks the group's scatter units (k_scatter: one per request run in the group;
// k_scatter_run: the single unit of an interval), finds each unit's first hit
// (Lemma lem:q, the p^2 start of Sec. 1.4, the mod-15015 or mod-15 wheel) and
// emits every hit of the unit into its warp's staging buffer in shared memory,
// counting hits per tile as it goes.  When a warp's buffer is full the CTA flushes: block scan of the
// per-tile counts, one atomic reservation per (tile, flush) in the tile's
// bucket (issued before the sort, consumed after it), each warp counting-sorts
// its own entries, and a store pass in which
// consecutive lanes write consecutive bucket slots.  Entries are the hit's bit
// offset inside its tile (uint32).  A bucket that would overflow its capacity
// spills to a global backstop list instead.
// ---------------------------------------------------------------------------
constexpr int kScT = 512, kScNW = kScT / 32, kScEW = 512, kScE = kScNW * kScEW;
constexpr uint32_t kCPT = kScatterMaxTiles / kScT;  // tile counters per thread in a flush
static_assert(kScatterMaxTiles % kScT == 0, "flush scan covers every tile");
constexpr size_t kScSmem = (size_t)kScE * 4 * 2 /*buf, srt*/ +
                           (size_t)kScatterMaxTiles * 4 * 4 /*tbase, tlim, gb, hist*/;

// Shared-memory layout of both scatter kernels.  Bucket slots are 32-bit entry
// offsets into the epoch's pool (its size is capped below 2^32 entries).
struct ScShared {
    uint32_t *tbase, *tlim, *gb, *hist, *buf, *srt;
    __device__ explicit ScShared(unsigned char *raw)
    {
        tbase = reinterpret_cast<uint32_t *>(raw);
        tlim = tbase + kScatterMaxTiles;
        gb = tlim + kScatterMaxTiles;
        hist = gb + kScatterMaxTiles;
        buf = hist + kScatterMaxTiles;
        srt = buf + kScE;
    }
};

// bucket ranges of the group's tiles, per-tile counters zeroed
__device__ __forceinline__ void scatter_group_setup(const ScatterArgs &a, const GroupDesc &g, ScShared &sh)
{
    for (uint32_t k = threadIdx.x; k < g.ntiles; k += kScT) {
        const TileDesc &td = a.tiles[g.tile0 + k];
        sh.tbase[k] = (uint32_t)td.bkt_off;
        sh.tlim[k] = (uint32_t)td.bkt_off + td.bkt_cap;
        sh.hist[k] = 0;
    }
    __syncthreads();
}

// One flush of the CTA's staging buffers (every warp calls it after a barrier):
// block scan of the per-tile counts, one atomic reservation per non-empty tile
// (issued before the sort, consumed after it), a counting sort of each warp's
// entries by tile, and a store pass in which consecutive lanes write consecutive
// slots of one bucket.  Slots beyond a bucket's capacity go to the backstop list.
__device__ __forceinline__ void scatter_flush(const ScatterArgs &a, const GroupDesc &g, ScShared &sh,
                                              const uint32_t *wb, uint32_t wcnt, uint32_t *s_warp)
{
    const uint32_t tid = threadIdx.x, lane = tid & 31;
    const uint32_t bt = a.tile_log2, Bm = (1u << bt) - 1;
    // thread tid scans the counters of tiles [kCPT*tid, kCPT*tid + kCPT)
    const uint32_t k0 = kCPT * tid;
    uint32_t c[kCPT], r[kCPT], sum = 0;
#pragma unroll
    for (uint32_t j = 0; j < kCPT; ++j) {
        c[j] = k0 + j < g.ntiles ? sh.hist[k0 + j] : 0u;
        sum += c[j];
    }
    uint32_t total;
    const uint32_t ex = block_excl_scan<kScT>(sum, s_warp, &total);
    // the counters become sort cursors; one reservation per non-empty tile is
    // issued now and its result consumed after the sort
    uint32_t run = ex;
#pragma unroll
    for (uint32_t j = 0; j < kCPT; ++j) {
        r[j] = 0;
        if (k0 + j < g.ntiles) {
            sh.hist[k0 + j] = run;
            if (c[j]) r[j] = atomicAdd(&a.bkt_cnt[g.tile0 + k0 + j], c[j]);
        }
        run += c[j];
    }
    __syncthreads();
    for (uint32_t i = lane; i < wcnt; i += 32) {
        const uint32_t v = wb[i];
        sh.srt[atomicAdd(&sh.hist[v >> bt], 1u)] = v;
    }
    // sorted position i of tile k goes to slot gb[k] + i (32-bit, wrapping: the
    // sum lands in [tbase, tbase + reserved))
    run = ex;
#pragma unroll
    for (uint32_t j = 0; j < kCPT; ++j) {
        if (c[j]) sh.gb[k0 + j] = sh.tbase[k0 + j] + r[j] - run;
        run += c[j];
    }
    __syncthreads();
    for (uint32_t i = tid; i < total; i += kScT) {
        const uint32_t v = sh.srt[i];
        const uint32_t k = v >> bt;
        const uint32_t dst = sh.gb[k] + i;
        const uint32_t off = v & Bm;
        if (dst < sh.tlim[k]) {
            a.bkt[dst] = off;
        } else {
            const uint32_t o = atomicAdd(a.ovf_cnt, 1u);
            if (o < a.ovf_cap)
                a.ovf[o] = ((unsigned long long)(g.tile0 + k) << 32) | off;
            else
                atomicOr(a.err, kErrOverflow);
        }
    }
    // cursors are no longer read: zero the counts for the next round
    for (uint32_t k = tid; k < g.ntiles; k += kScT) sh.hist[k] = 0;
}

// BIG: the mod-15015 wheel (fewest hits; its first hit reads two tables);
// otherwise the mod-15 wheel (tables in registers: cheapest first hit)
template <bool BIG>
__global__ void __launch_bounds__(kScT, 2) k_scatter(ScatterArgs a)
{
    extern __shared__ __align__(16) unsigned char smraw[];
    ScShared sh(smraw);
    __shared__ uint32_t s_warp[33];

    const uint32_t tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const ChunkDesc ch = a.chunks[blockIdx.x];
    const uint32_t lo = ch.p_lo;
    const uint32_t bt = a.tile_log2;
    uint32_t *wb = sh.buf + warp * kScEW;

    for (uint32_t gi = 0; gi < a.ngroups; ++gi) {
        const GroupDesc g = a.groups[gi];
        if (lo >= min(ch.p_hi, g.p_hi)) continue;
        const uint32_t n = min(ch.p_hi, g.p_hi) - lo;
        const uint32_t nlg = (n + 31) / 32;
        const uint32_t su_end = g.su0 + g.nsu;
        scatter_group_setup(a, g, sh);

        uint32_t lg = warp, su = g.su0;
        bool need_load = true, need_hit = true, pf = false;
        uint32_t p = 0, h = kStateInf, s = 0, gw = 0, p_n = 0;
        uint64_t m = 0, m_n = 0;
        unsigned long long cs = 0, cs_n = 0;
        for (;;) {
            // ---- generate into the warp's staging buffer, counting per tile ----
            uint32_t wcnt = 0;
            bool full = false;
            while (lg < nlg) {
                if (need_load) {
                    // this lane group's prime, constant and carried state (prefetched
                    // while the previous lane group was emitting), then the next one's
                    const uint32_t idx = lg * 32 + lane;
                    if (pf) {
                        p = p_n;
                        m = m_n;
                        cs = cs_n;
                    } else {
                        p = idx < n ? a.primes[lo + idx] : 0u;
                        m = idx < n ? a.barrett[lo + idx] : 0ull;
                        cs = (g.carry_in && idx < n) ? a.carry[lo + idx - a.carry_base] : 0ull;
                    }
                    const uint32_t ni = (lg + kScNW) * 32 + lane;
                    pf = lg + kScNW < nlg;
                    if (pf) {
                        p_n = ni < n ? a.primes[lo + ni] : 0u;
                        m_n = ni < n ? a.barrett[lo + ni] : 0ull;
                        cs_n = (g.carry_in && ni < n) ? a.carry[lo + ni - a.carry_base] : 0ull;
                    }
                    need_load = false;
                }
                SUDesc u;
                if (need_hit) {
                    // first hits unit after unit; a unit in which no lane's prime has a
                    // hit (the common case: units shorter than the primes) is passed
                    // over here, without the emit path
                    const uint32_t idx = lg * 32 + lane;
                    for (;;) {
                        u = a.sus[su];
                        const bool cout = su + 1 == su_end && g.carry_out;
                        h = kStateInf;
                        s = 0;
                        if (su == g.su0 && g.carry_in) {
                            // continue from where this prime left the previous group
                            if (idx < n) {
                                h = (uint32_t)cs;
                                s = (uint32_t)(cs >> 32);
                            }
                        } else if (p != 0 && p <= u.plimit) {
                            // a first multiple already past the unit means no hit in it (the
                            // p^2 start and the wheel only move it later), unless the next
                            // hit has to be carried into the next group
                            const uint32_t q = lemma_q(u.J, p, m);
                            if (q < u.span || cout) {
                                const uint64_t hh = BIG ? first_hit_big_q(u.J, u.jw, p, q, a.wheel, s)
                                                        : first_hit_q(u.J, u.jw, p, q, s);
                                if (hh < kStateInf) h = (uint32_t)hh;
                            }
                        }
                        if (cout || __any_sync(0xffffffffu, h < u.span)) break;
                        if (++su == su_end) {
                            su = g.su0;
                            lg += kScNW;
                            need_load = true;
                            break;
                        }
                    }
                    if (need_load) continue;
                    gw = BIG ? __ldg(a.wheel.gapw + (s >> 3)) >> (4 * (s & 7)) : 0u;
                    need_hit = false;
                } else {
                    u = a.sus[su];
                }
                const uint32_t ebase = u.tile_rel << bt;
                for (;;) {
                    const bool act = h < u.span;
                    const uint32_t mask = __ballot_sync(0xffffffffu, act);
                    if (!mask) break;
                    if (wcnt + 32 > (uint32_t)kScEW) {
                        full = true;
                        break;
                    }
                    if (act) {
                        const uint32_t v = ebase + h;
                        wb[wcnt + __popc(mask & lanemask_lt())] = v;
                        atomicAdd(&sh.hist[v >> bt], 1u);
                        if (BIG) {
                            const uint64_t nh = (uint64_t)h + (uint64_t)(gw & 15u) * p;
                            h = nh >= kStateInf ? kStateInf : (uint32_t)nh;
                            gw >>= 4;
                            if (++s == kBigCycle) s = 0;
                            if ((s & 7) == 0) gw = __ldg(a.wheel.gapw + (s >> 3));
                        } else {
                            const uint64_t nh = (uint64_t)h + (uint64_t)wheel_gap(s) * p;
                            h = nh >= kStateInf ? kStateInf : (uint32_t)nh;
                            s = (s + 1) & 7;
                        }
                    }
                    wcnt += __popc(mask);
                }
                if (full) break;
                need_hit = true;
                if (su + 1 == su_end && g.carry_out) {
                    // the next group starts where this unit ends: keep the next hit
                    // (the host carries only inside epochs of at most 2^32 bits, so a
                    // saturated next hit lies beyond the epoch)
                    const uint32_t idx = lg * 32 + lane;
                    if (idx < n)
                        a.carry[lo + idx - a.carry_base] =
                            ((unsigned long long)s << 32) | (h == kStateInf ? kStateInf : h - u.span);
                }
                if (++su == su_end) {
                    su = g.su0;
                    lg += kScNW;
                    need_load = true;
                }
            }
            const bool more = lg < nlg;
            __syncthreads();
            scatter_flush(a, g, sh, wb, wcnt, s_warp);
            if (!__syncthreads_or(more)) break;
        }
    }
}

// ---------------------------------------------------------------------------
// Scatter of a single request (one contiguous interval): every group is one
// scatter unit and starts where the previous one ends, across epochs too, so
// each large prime keeps one 64-bit state word for the whole interval -- its
// next hit relative to the start of the next group to be scattered (48 bits;
// all ones = none left) and its wheel position (16 bits).  First hits (Lemma
// lem:q, the p^2 start of Sec. 1.4, the wheel) are computed once, by the first
// group of the interval; every later visit reads the word, emits the prime's
// hits in the group and writes the word back.  Lanes past the chunk's end load
// padding and stay idle.
// ---------------------------------------------------------------------------
constexpr unsigned long long kRunInf = (1ull << 48) - 1;

// One wheel step of a large prime: the next struck multiple.  Mod-15015 wheel:
// gw holds the unused gaps (4 bits each, 1..11, never 0) of gap word gwi, so an
// empty word means all 8 are used; mod-15 wheel: s is the cycle position.
template <bool BIG>
__device__ __forceinline__ void scatter_step(uint64_t &h, uint32_t &s, uint32_t &gw, uint32_t &gwi, uint32_t p,
                                             const uint32_t *gapw)
{
    if (BIG) {
        h += (uint64_t)(gw & 15u) * p;
        gw >>= 4;
        if (gw == 0) {
            gwi = gwi + 1 == kBigWords ? 0u : gwi + 1;
            gw = __ldg(gapw + gwi);
        }
    } else {
        h += (uint64_t)wheel_gap(s) * p;
        s = (s + 1) & 7;
    }
}

// mod-15015 cycle position of a prime whose gap word gwi has the gaps gw left
__device__ __forceinline__ uint32_t big_wheel_pos(uint32_t gw, uint32_t gwi)
{
    return 8 * gwi + 8 - ((32 - __clz(gw) + 3) >> 2);
}

// Loads of words read once per launch (a chunk's primes, Barrett constants and state
// words), marked not to allocate in L1: the L1 then keeps what is read again and again,
// the mod-15015 wheel tables of the first hits and the gap words of the emission.
__device__ __forceinline__ uint32_t ld_no_l1_alloc_u32(const uint32_t *p)
{
    uint32_t v;
    asm volatile("ld.global.L1::no_allocate.u32 %0, [%1];" : "=r"(v) : "l"(p));
    return v;
}
__device__ __forceinline__ unsigned long long ld_no_l1_alloc_u64(const void *p)
{
    unsigned long long v;
    asm volatile("ld.global.L1::no_allocate.u64 %0, [%1];" : "=l"(v) : "l"(p));
    return v;
}

template <bool BIG>
__global__ void __launch_bounds__(kScT, 2) k_scatter_run(ScatterArgs a)
{
    extern __shared__ __align__(16) unsigned char smraw[];
    ScShared sh(smraw);
    __shared__ uint32_t s_warp[33];

    const uint32_t tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const uint32_t lt = lanemask_lt();
    const ChunkDesc ch = a.chunks[blockIdx.x];
    const uint32_t n = ch.p_hi - ch.p_lo;  // every group covers the chunk's primes
    const uint32_t nlg = (n + 31) / 32;
    const uint32_t bt = a.tile_log2;
    const uint32_t *pr = a.primes + ch.p_lo;
    const uint64_t *pm = a.barrett + ch.p_lo;
    unsigned long long *stw = a.state + (ch.p_lo - a.state_base);
    uint32_t *wb = sh.buf + warp * kScEW;

    for (uint32_t gi = 0; gi < a.ngroups; ++gi) {
        const GroupDesc g = a.groups[gi];
        const SUDesc u = a.sus[g.su0];
        const bool first = a.run_first && gi == 0;
        const bool last = a.run_last && gi + 1 == a.ngroups;  // nothing reads the state after it
        const uint32_t span = u.span, ebase = u.tile_rel << bt;
        const uint32_t jsx = u.jw;
        scatter_group_setup(a, g, sh);

        // the lane group's prime and state (one prime per lane)
        uint32_t lg = warp, p = 0, s = 0, gw = 0, idx = 0, gwi = 0;
        uint64_t h = 0;
        // the next lane group's words, loaded ahead: its prime and either its state
        // word or, for a prime that takes a first hit in the interval's first group, its
        // Barrett constant (the primes are padded past the chunk, the constants are not)
        // Whether the chunk's primes take first hits is decided per chunk (a warp-uniform
        // choice of one load); only the chunk that straddles a streamed interval's
        // boundary decides per prime.
        const uint32_t rel0 = ch.p_lo - a.state_base;  // index of the chunk's first prime in the state
        const bool all_fresh = first && rel0 >= a.first_from;
        const bool mixed = first && !all_fresh && rel0 + n > a.first_from;
        auto fresh = [&](uint32_t i) { return all_fresh || (mixed && rel0 + i >= a.first_from); };
        auto next_word = [&](uint32_t i) -> unsigned long long {
            if (all_fresh) return i < n ? ld_no_l1_alloc_u64(pm + i) : 0ull;
            if (!mixed) return ld_no_l1_alloc_u64(stw + i);
            return rel0 + i >= a.first_from ? (i < n ? ld_no_l1_alloc_u64(pm + i) : 0ull)
                                            : ld_no_l1_alloc_u64(stw + i);
        };
        uint32_t p_n = 0;
        unsigned long long w_n = 0;
        if (lg < nlg) {
            const uint32_t ni = lg * 32 + lane;
            p_n = ld_no_l1_alloc_u32(pr + ni);
            w_n = next_word(ni);
        }
        bool need = true;
        for (;;) {
            uint32_t wcnt = 0;
            bool full = false;
            while (lg < nlg) {
                if (need) {
                    idx = lg * 32 + lane;
                    p = p_n;
                    const unsigned long long w = w_n;
                    const uint32_t nl = lg + kScNW;
                    if (nl < nlg) {
                        const uint32_t ni = nl * 32 + lane;
                        p_n = ld_no_l1_alloc_u32(pr + ni);
                        w_n = next_word(ni);
                    }
                    h = kRunInf;
                    s = 0;
                    if (idx < n) {
                        if (fresh(idx)) {
                            if (p <= u.plimit) {
                                const uint64_t hh = BIG ? first_hit_big(u.J, jsx, p, w, a.wheel, s)
                                                        : first_hit(u.J, jsx, p, w, s);
                                h = hh < kRunInf ? hh : kRunInf;
                            }
                        } else {
                            h = w & kRunInf;
                            s = (uint32_t)(w >> 48);
                        }
                    }
                    gwi = s >> 3;
                    gw = (BIG && h < span) ? __ldg(a.wheel.gapw + gwi) >> (4 * (s & 7)) : 0u;
                    need = false;
                }
                for (;;) {
                    const bool act = h < span;
                    const uint32_t mask = __ballot_sync(0xffffffffu, act);
                    if (!mask) break;
                    if (wcnt + 32 > (uint32_t)kScEW) {
                        full = true;
                        break;
                    }
                    if (act) {
                        const uint32_t v = ebase + (uint32_t)h;
                        wb[wcnt + __popc(mask & lt)] = v;
                        atomicAdd(&sh.hist[v >> bt], 1u);
                        scatter_step<BIG>(h, s, gw, gwi, p, a.wheel.gapw);
                    }
                    wcnt += __popc(mask);
                }
                if (full) break;
                // next hit relative to the next group (h < span + 11 p < 2^48 unless none)
                // with the wheel position (a lane that emitted nothing kept its own)
                if (BIG && gw) s = big_wheel_pos(gw, gwi);
                if (idx < n && !last) stw[idx] = ((unsigned long long)s << 48) | (h == kRunInf ? kRunInf : h - span);
                lg += kScNW;
                need = true;
            }
            __syncthreads();
            scatter_flush(a, g, sh, wb, wcnt, s_warp);
            if (!__syncthreads_or(lg < nlg)) break;
        }
    }
}

cudaError_t launch_scatter(const ScatterArgs &a, uint32_t nchunks, bool big_wheel, bool run, cudaStream_t st)
{
    if (run) {
        if (big_wheel)
            k_scatter_run<true><<<nchunks, kScT, kScSmem, st>>>(a);
        else
            k_scatter_run<false><<<nchunks, kScT, kScSmem, st>>>(a);
    } else {
        if (big_wheel)
            k_scatter<true><<<nchunks, kScT, kScSmem, st>>>(a);
        else
            k_scatter<false><<<nchunks, kScT, kScSmem, st>>>(a);
    }
    return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// base of Sec. 1.4 on the device
// ---------------------------------------------------------------------------
// odd primes below 2^17 (index j < 2^16 stands for 2j+1), one CTA: striking with
// every odd d <= 361 = floor(sqrt(131071)) from d^2 on (Sec. 1.1, Sec. 1.4)
__global__ void __launch_bounds__(1024) k_bootstrap(uint32_t *primes_out, uint32_t *count_out)
{
    __shared__ uint32_t bits[2048];
    __shared__ uint32_t s_warp[33];
    const uint32_t tid = threadIdx.x;
    for (uint32_t i = tid; i < 2048; i += 1024) bits[i] = 0;
    __syncthreads();
    if (tid < 180) {
        const uint32_t d = 2 * tid + 3;
        for (uint32_t j = (d * d - 1) / 2; j < 65536; j += d) atomicOr(&bits[j >> 5], 1u << (j & 31));
    }
    __syncthreads();
    uint32_t w0 = ~bits[2 * tid], w1 = ~bits[2 * tid + 1];
    if (tid == 0) w0 &= ~1u;  // the number 1
    uint32_t tot;
    uint32_t pos = block_excl_scan<1024>(__popc(w0) + __popc(w1), s_warp, &tot);
    while (w0) {
        const uint32_t b = __ffs(w0) - 1;
        w0 &= w0 - 1;
        primes_out[pos++] = 2 * (64 * tid + b) + 1;
    }
    while (w1) {
        const uint32_t b = __ffs(w1) - 1;
        w1 &= w1 - 1;
        primes_out[pos++] = 2 * (64 * tid + 32 + b) + 1;
    }
    if (tid == 0) *count_out = tot;
}

constexpr int kCpT = 1024, kCpW = 4;  // compaction: threads per block, words per thread

// zero bits of word w among valid indices 1..jmax
__device__ __forceinline__ uint32_t prime_bits(const uint32_t *bits, uint64_t w, uint64_t nwords,
                                               uint64_t jmax)
{
    if (w >= nwords) return 0;
    uint32_t v = ~bits[w];
    if (w == 0) v &= ~1u;
    const uint64_t j = 32 * w;
    if (j > jmax) return 0;
    if (jmax - j < 31) v &= (1u << (jmax - j + 1)) - 1;
    return v;
}

__global__ void __launch_bounds__(kCpT) k_compact_count(const uint32_t *bits, uint64_t nwords, uint64_t jmax,
                                                        uint32_t *block_cnt)
{
    __shared__ uint32_t s_warp[33];
    const uint64_t w0 = ((uint64_t)blockIdx.x * kCpT + threadIdx.x) * kCpW;
    uint32_t c = 0;
    for (int k = 0; k < kCpW; ++k) c += __popc(prime_bits(bits, w0 + k, nwords, jmax));
    uint32_t tot;
    block_excl_scan<kCpT>(c, s_warp, &tot);
    if (threadIdx.x == 0) block_cnt[blockIdx.x] = tot;
}

__global__ void __launch_bounds__(1024) k_compact_scan(const uint32_t *block_cnt, uint32_t nblocks,
                                                       uint32_t *block_off, uint32_t *total)
{
    __shared__ uint32_t s_warp[33];
    const uint32_t per = (nblocks + 1023) / 1024;
    const uint32_t base = threadIdx.x * per;
    uint32_t sum = 0;
    for (uint32_t k = 0; k < per; ++k)
        if (base + k < nblocks) sum += block_cnt[base + k];
    uint32_t tot;
    uint32_t run = block_excl_scan<1024>(sum, s_warp, &tot);
    for (uint32_t k = 0; k < per; ++k) {
        if (base + k < nblocks) {
            block_off[base + k] = run;
            run += block_cnt[base + k];
        }
    }
    if (threadIdx.x == 0) *total = tot;
}

__global__ void __launch_bounds__(kCpT) k_compact_write(const uint32_t *bits, uint64_t nwords, uint64_t jmax,
                                                        const uint32_t *block_off, uint32_t *primes_out,
                                                        uint64_t cap)
{
    __shared__ uint32_t s_warp[33];
    const uint64_t w0 = ((uint64_t)blockIdx.x * kCpT + threadIdx.x) * kCpW;
    uint32_t v[kCpW];
    uint32_t c = 0;
    for (int k = 0; k < kCpW; ++k) {
        v[k] = prime_bits(bits, w0 + k, nwords, jmax);
        c += __popc(v[k]);
    }
    uint32_t tot;
    uint32_t pos = block_off[blockIdx.x] + block_excl_scan<kCpT>(c, s_warp, &tot);
    for (int k = 0; k < kCpW; ++k) {
        uint32_t x = v[k];
        while (x) {
            const uint32_t b = __ffs(x) - 1;
            x &= x - 1;
            // never past the buffer: the host rejects a count above its capacity
            if (pos < cap) primes_out[pos] = (uint32_t)(2 * (32 * (w0 + k) + b) + 1);
            ++pos;
        }
    }
}

cudaError_t launch_bootstrap(uint32_t *primes_out, uint32_t *count_out, cudaStream_t st)
{
    k_bootstrap<<<1, 1024, 0, st>>>(primes_out, count_out);
    return cudaGetLastError();
}

cudaError_t launch_compact(const uint32_t *bits, uint64_t nbits, uint64_t jmax, uint32_t *block_cnt,
                           uint32_t *block_off, uint32_t *primes_out, uint64_t cap, uint32_t *total_out,
                           cudaStream_t st)
{
    const uint64_t nwords = nbits / 32;
    const uint32_t nblocks = (uint32_t)((nwords + (uint64_t)kCpT * kCpW - 1) / ((uint64_t)kCpT * kCpW));
    k_compact_count<<<nblocks, kCpT, 0, st>>>(bits, nwords, jmax, block_cnt);
    k_compact_scan<<<1, 1024, 0, st>>>(block_cnt, nblocks, block_off, total_out);
    if (primes_out) k_compact_write<<<nblocks, kCpT, 0, st>>>(bits, nwords, jmax, block_off, primes_out, cap);
    return cudaGetLastError();
}

__global__ void k_barrett(const uint32_t *primes, uint64_t n, uint64_t *m)
{
    for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (uint64_t)gridDim.x * blockDim.x)
        m[i] = 0xFFFFFFFFFFFFFFFFull / primes[i];
}

cudaError_t launch_barrett(const uint32_t *primes, uint64_t n, uint64_t *m, cudaStream_t st)
{
    k_barrett<<<1024, 256, 0, st>>>(primes, n, m);
    return cudaGetLastError();
}

// sum of n uint32 counters into *acc (profiling: exact large-prime hit count)
__global__ void k_sum_u32(const uint32_t *v, uint32_t n, unsigned long long *acc)
{
    unsigned long long c = 0;
    for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) c += v[i];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) c += __shfl_xor_sync(0xffffffffu, c, o);
    if ((threadIdx.x & 31) == 0 && c) atomicAdd(acc, c);
}

cudaError_t launch_sum_u32(const uint32_t *v, uint32_t n, unsigned long long *acc, cudaStream_t st)
{
    k_sum_u32<<<64, 256, 0, st>>>(v, n, acc);
    return cudaGetLastError();
}

// twin pairs straddling tiles t and t+1 of one interval (count mode): the last bit of
// tile t and the first bit of tile t+1 both primes; the pair belongs to the segment of
// its lower member
__global__ void k_seg_edges(const TileDesc *tiles, const uint8_t *edge, uint32_t ntiles, uint64_t seg_j0,
                            uint32_t seg_l, unsigned long long *seg_twins)
{
    for (uint32_t t = blockIdx.x * blockDim.x + threadIdx.x; t + 1 < ntiles; t += gridDim.x * blockDim.x) {
        const TileDesc a = tiles[t];
        if (a.J + a.len == tiles[t + 1].J && (edge[t] & 2) && (edge[t + 1] & 1))
            atomicAdd(&seg_twins[(a.J + a.len - 1 - seg_j0) >> seg_l], 1ull);
    }
}

cudaError_t launch_seg_edges(const TileDesc *tiles, const uint8_t *edge, uint32_t ntiles, uint64_t seg_j0,
                             uint32_t seg_l, unsigned long long *seg_twins, cudaStream_t st)
{
    if (ntiles > 1) k_seg_edges<<<(ntiles + 255) / 256 < 1024 ? (ntiles + 255) / 256 : 1024, 256, 0, st>>>(
        tiles, edge, ntiles, seg_j0, seg_l, seg_twins);
    return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// Goldbach search (Sec. 5: verifying the Goldbach conjecture is what the table is
// made for).  For an even N and an odd prime p, N - p = 2J + 1 with J = N/2 - (p+1)/2,
// so for 32 consecutive even numbers N_i = N_0 + 2i the candidates N_i - p are the 32
// consecutive table bits from J_0 = N_0/2 - (p+1)/2 on: one 32-bit window of the table
// (two words and a funnel shift) answers "is N_i - p prime" for all 32 at once (bit 0
// = prime; the number 1, J = 0, is masked out).  Thread b takes N_i = n_lo + 2(32b + i)
// and tries p = 3, 5, 7, ... in order, marking each number done at the first p whose
// window bit is 0, so that p is its smallest partition prime.  It stops when all its
// numbers are done, the primes run out, or the windows fall below the table (only
// when the table starts at 1: then J < 0 means p > N - 1 and the number fails).  The
// largest minimal p among its numbers is the p that completed the last of them, the
// first N attaining it the lowest of the numbers completed by that p.
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(256) k_goldbach(const uint32_t *__restrict__ bits, uint64_t j0, uint64_t nwords,
                                                  const uint32_t *__restrict__ primes, uint32_t nprimes,
                                                  uint64_t n_lo, uint64_t count, uint32_t win_log2,
                                                  GoldbachWindow *out)
{
    const uint32_t lane = threadIdx.x & 31;
    const uint64_t nblk = (count + 31) / 32;
    const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;  // a multiple of 32
    // whole warps walk the blocks together (b - lane is the same for the 32 lanes), so
    // the shuffles below are warp-uniform
    for (uint64_t b = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; b - lane < nblk; b += stride) {
        // valid: the block's numbers (fewer in the last block); alive: those that can
        // still be done; done: those whose smallest partition prime has been found
        uint32_t valid = 0, alive = 0, done = 0, p_last = 0, first_last = 0;
        if (b < nblk) {
            const uint64_t left = count - 32 * b;
            valid = alive = left >= 32 ? 0xFFFFFFFFu : (1u << left) - 1u;
            const int64_t hN = (int64_t)((n_lo >> 1) + 32 * b);  // N_0 / 2 (numbers below 2^63)
            const int64_t base = hN - (int64_t)j0;               // relative J of N_0 - 1
            // Away from the table's edges (every block unless the table starts at 1, and
            // every block but the last): for p = 2q - 1 the window starts at relative
            // J = base - q, i.e. word (base >> 5) + ((bb - q) >> 5), bit (bb - q) & 31 with
            // bb = base & 31, all in 32-bit arithmetic.  The host guarantees base - q >= 0
            // for every p <= p_max when j0 > 0, and the hi word exists except near the end.
            const bool edges = j0 == 0 || (uint64_t)(base >> 5) + 1 >= nwords;
            if (!edges) {
                const uint32_t *row = bits + (base >> 5);
                const int32_t bb = (int32_t)(base & 31);
                for (uint32_t k = 0; k < nprimes && (alive & ~done); ++k) {
                    const uint32_t p = __ldg(primes + k);
                    const int32_t t = bb - (int32_t)((p + 1) >> 1);
                    const uint32_t *r = row + (t >> 5);  // arithmetic shift: floor division
                    const uint32_t w = __funnelshift_r(__ldg(r), __ldg(r + 1), (uint32_t)t & 31);
                    const uint32_t prime = ~w & alive & ~done;
                    if (prime) {
                        done |= prime;
                        p_last = p;
                        first_last = __ffs(prime) - 1;
                    }
                }
            } else {
                for (uint32_t k = 0; k < nprimes && (alive & ~done); ++k) {
                    const uint32_t p = __ldg(primes + k);
                    const int64_t Jw = hN - (int64_t)((p + 1) >> 1);  // J of N_0 - p
                    const int64_t jw = Jw - (int64_t)j0;               // relative to the table
                    uint32_t w;
                    if (jw >= 0) {
                        const uint64_t q = (uint64_t)jw >> 5;
                        const uint32_t lo = __ldg(bits + q);
                        const uint32_t hi = q + 1 < nwords ? __ldg(bits + q + 1) : 0xFFFFFFFFu;
                        w = __funnelshift_r(lo, hi, (uint32_t)jw & 31);
                    } else {
                        // only when the table starts at 1 (j0 = 0): numbers i < -jw have
                        // N_i - p < 1, and so for every larger p: they fail
                        if (jw <= -32) break;
                        const uint32_t sh = (uint32_t)(-jw), below = (1u << sh) - 1u;
                        w = (__ldg(bits) << sh) | below;
                        alive &= ~below | done;
                    }
                    uint32_t prime = ~w & alive & ~done;
                    if (Jw <= 0 && Jw > -32) prime &= ~(1u << (uint32_t)(-Jw));  // N_i - p = 1
                    if (prime) {
                        done |= prime;
                        p_last = p;
                        first_last = __ffs(prime) - 1;
                    }
                }
            }
        }
        const uint32_t fail = __popc(valid & ~done);
        const uint64_t off = (32 * b + first_last) & ((1ull << win_log2) - 1);
        unsigned long long key = p_last ? ((unsigned long long)p_last << 32) | (0xFFFFFFFFull - off) : 0ull;
        if (win_log2 >= 10) {
            // a warp's 32 blocks (1024 numbers) lie in one window
            uint32_t f = fail;
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) {
                const unsigned long long kk = __shfl_xor_sync(0xffffffffu, key, o);
                key = kk > key ? kk : key;
                f += __shfl_xor_sync(0xffffffffu, f, o);
            }
            if (lane == 0) {
                GoldbachWindow &wd = out[(32 * (b - lane)) >> win_log2];
                if (key) atomicMax(&wd.key, key);
                if (f) atomicAdd(&wd.failures, (unsigned long long)f);
            }
        } else if (b < nblk) {
            // a block's 32 numbers lie in one window (win_log2 >= 5)
            GoldbachWindow &wd = out[(32 * b) >> win_log2];
            if (key) atomicMax(&wd.key, key);
            if (fail) atomicAdd(&wd.failures, (unsigned long long)fail);
        }
    }
}

cudaError_t launch_goldbach(const uint32_t *bits, uint64_t j0, uint64_t nwords, const uint32_t *primes,
                            uint32_t nprimes, uint64_t n_lo, uint64_t count, uint32_t win_log2, GoldbachWindow *out,
                            int nsm, cudaStream_t st)
{
    const uint64_t want = ((count + 31) / 32 + 255) / 256;  // one thread per 32 even numbers
    const uint32_t grid = (uint32_t)(want < (uint64_t)nsm * 8 ? want : (uint64_t)nsm * 8);
    if (grid) k_goldbach<<<grid, 256, 0, st>>>(bits, j0, nwords, primes, nprimes, n_lo, count, win_log2, out);
    return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// popcount of a table
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(512) k_popcount(const uint32_t *words, uint64_t nwords, unsigned long long *acc)
{
    unsigned long long c = 0;
    const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
    const uint64_t i0 = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if ((reinterpret_cast<uintptr_t>(words) & 15) == 0) {
        const uint4 *w4 = reinterpret_cast<const uint4 *>(words);
        const uint64_t n4 = nwords / 4;
        for (uint64_t i = i0; i < n4; i += stride) {
            const uint4 v = __ldcs(w4 + i);
            c += __popc(v.x) + __popc(v.y) + __popc(v.z) + __popc(v.w);
        }
        for (uint64_t i = 4 * n4 + i0; i < nwords; i += stride) c += __popc(words[i]);
    } else {
        for (uint64_t i = i0; i < nwords; i += stride) c += __popc(words[i]);
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) c += __shfl_xor_sync(0xffffffffu, c, o);
    if ((threadIdx.x & 31) == 0 && c) atomicAdd(acc, c);
}

cudaError_t launch_popcount(const uint32_t *words, uint64_t nwords, unsigned long long *acc, uint32_t grid,
                            cudaStream_t st)
{
    k_popcount<<<grid, 512, 0, st>>>(words, nwords, acc);
    return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// shared-memory atomic OR rate: a stream of conflict-free atomics with almost no
// other instructions.  Lane k of a warp always addresses bank k (word row*32 + k),
// and the rows are immediate offsets from one register, so the unrolled body is
// one ATOMS per atomic and the loop adds two instructions per 64 atomics: the
// kernel is bound by the shared-memory atomic unit, not by instruction issue.
// ---------------------------------------------------------------------------
constexpr int kProbeWords = 32768;  // 128 KB, the size of a 2^20-bit tile
constexpr int kProbeUnroll = 64;    // atomics per loop trip (64 rows of 32 words)
constexpr int kProbeTrips = 64;     // loop trips per thread

__global__ void __launch_bounds__(1024) k_probe_smem(uint32_t *sink)
{
    extern __shared__ uint32_t pm[];
    for (uint32_t i = threadIdx.x; i < kProbeWords; i += blockDim.x) pm[i] = 0;
    __syncthreads();
    const uint32_t lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    // warp w works on rows 64*(w%16) .. +63 (a 32 KB-wide stripe per warp pair); bit
    // values differ by thread so the table's final contents depend on every atomic
    uint32_t *base = pm + (kProbeUnroll * 32) * (warp & 15) + lane;
    const uint32_t bit = 1u << ((threadIdx.x * 7u + blockIdx.x) & 31);
    for (int it = 0; it < kProbeTrips; ++it) {
#pragma unroll
        for (int k = 0; k < kProbeUnroll; ++k) atomicOr(base + 32 * k, bit);
    }
    __syncthreads();
    uint32_t v = 0;
    for (uint32_t i = threadIdx.x; i < kProbeWords; i += blockDim.x) v ^= pm[i];
    if (v == 0x12345678u) sink[0] = v;  // keeps the work observable
}

cudaError_t probe_smem_atomics(int nsm, double *atom_per_s)
{
    uint32_t *sink = nullptr;
    cudaError_t e = cudaMalloc(&sink, 16);
    if (e != cudaSuccess) return e;
    const size_t smem = (size_t)kProbeWords * 4;
    cudaFuncSetAttribute(k_probe_smem, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    cudaEvent_t a, b;
    cudaEventCreate(&a);
    cudaEventCreate(&b);
    const int grid = nsm;
    k_probe_smem<<<grid, 1024, smem>>>(sink);  // warm-up
    cudaEventRecord(a);
    const int reps = 5;
    for (int r = 0; r < reps; ++r) k_probe_smem<<<grid, 1024, smem>>>(sink);
    cudaEventRecord(b);
    e = cudaEventSynchronize(b);
    float ms = 0;
    cudaEventElapsedTime(&ms, a, b);
    if (e == cudaSuccess) e = cudaGetLastError();
    *atom_per_s = (double)grid * 1024.0 * kProbeTrips * kProbeUnroll * reps / (ms * 1e-3);
    cudaEventDestroy(a);
    cudaEventDestroy(b);
    cudaFree(sink);
    return e;
}

// ---------------------------------------------------------------------------
// distributed shared memory OR rate: clusters of C CTAs, every thread a stream of
// conflict-free ORs into a cluster rank's shared memory through the cluster window
// (mapa + red.shared::cluster), target = own rank (peer = 0) or the next rank (peer =
// 1).  Cluster barriers at the start (every slice zeroed and every CTA running before
// any remote access) and at the end (no remote access after a CTA may exit), reached
// by every thread of every CTA.
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(1024, 1) k_probe_dsmem(uint32_t *sink, int peer)
{
    extern __shared__ uint32_t pm[];
    for (uint32_t i = threadIdx.x; i < kProbeWords; i += blockDim.x) pm[i] = 0;
    cluster_barrier();
    const uint32_t lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const uint32_t bit = 1u << ((threadIdx.x * 7u + blockIdx.x) & 31);
    const uint32_t tgt = peer ? (cluster_rank() + 1) % cluster_size() : cluster_rank();
    uint32_t base;
    const uint32_t local = (uint32_t)__cvta_generic_to_shared(pm + (kProbeUnroll * 32) * (warp & 15) + lane);
    asm volatile("mapa.shared::cluster.u32 %0, %1, %2;" : "=r"(base) : "r"(local), "r"(tgt));
    for (int it = 0; it < kProbeTrips; ++it) {
#pragma unroll
        for (int k = 0; k < kProbeUnroll; ++k)
            asm volatile("red.relaxed.cluster.shared::cluster.or.b32 [%0], %1;" ::"r"(base + 128u * k), "r"(bit)
                         : "memory");
    }
    cluster_barrier();
    uint32_t v = 0;
    for (uint32_t i = threadIdx.x; i < kProbeWords; i += blockDim.x) v ^= pm[i];
    if (v == 0x12345678u) sink[0] = v;
}

cudaError_t probe_dsmem_atomics(uint32_t csize, int peer, double *atom_per_s, uint32_t *ctas)
{
    uint32_t *sink = nullptr;
    cudaError_t e = cudaMalloc(&sink, 16);
    if (e != cudaSuccess) return e;
    const size_t smem = (size_t)kProbeWords * 4;
    cudaFuncSetAttribute(k_probe_dsmem, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeClusterDimension;
    at[0].val.clusterDim.x = csize;
    at[0].val.clusterDim.y = 1;
    at[0].val.clusterDim.z = 1;
    cudaLaunchConfig_t cfg = {};
    cfg.blockDim = dim3(1024);
    cfg.gridDim = dim3(csize);
    cfg.dynamicSmemBytes = smem;
    cfg.attrs = at;
    cfg.numAttrs = 1;
    int ncl = 0;
    e = cudaOccupancyMaxActiveClusters(&ncl, k_probe_dsmem, &cfg);
    if (e == cudaSuccess && ncl < 1) e = cudaErrorInvalidConfiguration;
    float ms = 0;
    if (e == cudaSuccess) {
        cfg.gridDim = dim3(ncl * csize);
        cudaEvent_t a, b;
        cudaEventCreate(&a);
        cudaEventCreate(&b);
        e = cudaLaunchKernelEx(&cfg, k_probe_dsmem, sink, peer);  // warm-up
        cudaEventRecord(a);
        for (int r = 0; r < 5 && e == cudaSuccess; ++r) e = cudaLaunchKernelEx(&cfg, k_probe_dsmem, sink, peer);
        cudaEventRecord(b);
        if (e == cudaSuccess) e = cudaEventSynchronize(b);
        cudaEventElapsedTime(&ms, a, b);
        cudaEventDestroy(a);
        cudaEventDestroy(b);
    }
    if (e == cudaSuccess) {
        *atom_per_s = (double)ncl * csize * 1024.0 * kProbeTrips * kProbeUnroll * 5 / (ms * 1e-3);
        *ctas = (uint32_t)(ncl * csize);
    }
    cudaFree(sink);
    return e;
}

cudaError_t set_kernel_attributes()
{
    const int big = (int)tile_smem_bytes(20);
    cudaError_t e = cudaFuncSetAttribute(k_tile<1024>, cudaFuncAttributeMaxDynamicSharedMemorySize, big);
    if (e == cudaSuccess) e = cudaFuncSetAttribute(k_tile<512>, cudaFuncAttributeMaxDynamicSharedMemorySize, big);
    if (e == cudaSuccess) e = cudaFuncSetAttribute(k_tile<256>, cudaFuncAttributeMaxDynamicSharedMemorySize, big);
    if (e == cudaSuccess) e = cudaFuncSetAttribute(k_ctile<2>, cudaFuncAttributeMaxDynamicSharedMemorySize, big);
    if (e == cudaSuccess) e = cudaFuncSetAttribute(k_scatter<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kScSmem);
    if (e == cudaSuccess) e = cudaFuncSetAttribute(k_scatter<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kScSmem);
    if (e == cudaSuccess) e = cudaFuncSetAttribute(k_scatter_run<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kScSmem);
    if (e == cudaSuccess) e = cudaFuncSetAttribute(k_scatter_run<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kScSmem);
    return e;
}

}  // namespace gbs
