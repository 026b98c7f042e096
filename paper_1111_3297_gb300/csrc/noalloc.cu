// Composite count of a sieve table without any device allocation.
//
// sieve_count needs a context, whose device buffers (including the count
// accumulator) are allocated with cudaMalloc.  Some callers cannot allocate:
// code running under another framework's memory manager that has reserved the
// device's memory for its own pool, and latency-critical callers that must not
// hit the implicit device synchronisation cudaMalloc/cudaFree can cause.  This
// entry point needs neither a context nor an allocation: its only scratch is a
// fixed array of per-block partial counts in this file, resolved once per device.
#include "gbsieve.h"

#include <cuda_runtime.h>
#include <mutex>

namespace {

constexpr uint32_t kPartialsMax = 65536;        // blocks of the first pass (the scratch size)
constexpr uint64_t kWordsPerBlock = 1ull << 16; // words each first-pass block counts
static_assert((uint64_t)kPartialsMax * kWordsPerBlock * 32 == SIEVE_NOALLOC_MAX_BITS, "size limit");

// One partial count per first-pass block.  Every GPU that loads this library
// holds these 512 KB until the process exits.  In host code this name is only a
// host-side stand-in; kernels get the device address resolved below.
static __device__ __align__(256) unsigned long long g_partials[kPartialsMax];

constexpr int kMaxDevices = 256;
std::mutex g_mu;
unsigned long long *g_addr[kMaxDevices];  // device address of g_partials, per device

__global__ void __launch_bounds__(256) k_partials(const uint32_t *words, uint64_t nwords,
                                                 unsigned long long *part)
{
    const uint64_t w0 = (uint64_t)blockIdx.x * kWordsPerBlock;
    const uint64_t w1 = w0 + kWordsPerBlock < nwords ? w0 + kWordsPerBlock : nwords;
    unsigned long long c = 0;
    for (uint64_t i = w0 + threadIdx.x; i < w1; i += blockDim.x) c += __popc(words[i]);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) c += __shfl_xor_sync(0xffffffffu, c, o);
    __shared__ unsigned long long s[8];
    if ((threadIdx.x & 31) == 0) s[threadIdx.x >> 5] = c;
    __syncthreads();
    if (threadIdx.x == 0) {
        unsigned long long t = 0;
        for (int k = 0; k < 8; ++k) t += s[k];
        part[blockIdx.x] = t;  // every block overwrites its own entry: nothing needs clearing
    }
}

__global__ void __launch_bounds__(1024) k_total(const unsigned long long *part, uint32_t nblocks,
                                               unsigned long long *out)
{
    unsigned long long c = 0;
    for (uint32_t i = threadIdx.x; i < nblocks; i += blockDim.x) c += part[i];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) c += __shfl_xor_sync(0xffffffffu, c, o);
    __shared__ unsigned long long s[32];
    if ((threadIdx.x & 31) == 0) s[threadIdx.x >> 5] = c;
    __syncthreads();
    if (threadIdx.x == 0) {
        unsigned long long t = 0;
        for (int k = 0; k < 32; ++k) t += s[k];
        *out = t;
    }
}

}  // namespace

sieve_status sieve_count_noalloc(const uint32_t *dev_bits, uint64_t nbits, uint64_t *dev_count,
                                 sieve_stream stream)
{
    if (!dev_count || (nbits & 31) || (nbits && !dev_bits)) return SIEVE_EINVAL;
    if (nbits > SIEVE_NOALLOC_MAX_BITS) return SIEVE_ERANGE;
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) return SIEVE_ECUDA;
    unsigned long long *part;
    {
        // set-up, once per device, with that device current
        std::lock_guard<std::mutex> g(g_mu);
        if (!g_addr[dev]) {
            void *p = nullptr;
            if (cudaGetSymbolAddress(&p, g_partials) != cudaSuccess || !p) {
                cudaGetLastError();
                return SIEVE_ECUDA;
            }
            g_addr[dev] = static_cast<unsigned long long *>(p);
        }
        part = g_addr[dev];
    }
    const uint64_t nwords = nbits / 32;
    const uint32_t nblocks = (uint32_t)((nwords + kWordsPerBlock - 1) / kWordsPerBlock);
    cudaStream_t st = (cudaStream_t)stream;
    if (nblocks) k_partials<<<nblocks, 256, 0, st>>>(dev_bits, nwords, part);
    k_total<<<1, 1024, 0, st>>>(part, nblocks, (unsigned long long *)dev_count);
    return cudaGetLastError() == cudaSuccess ? SIEVE_OK : SIEVE_ECUDA;
}
