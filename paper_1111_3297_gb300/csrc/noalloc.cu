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
#include "host_internal.h"

#include <cstdio>
#include <cuda.h>
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
unsigned long long g_ctx_id[kMaxDevices]; // id of the context that address belongs to

// Unique id of the current context (cuCtxGetId through the runtime's driver entry
// points, so no link against libcuda).  A device reset destroys the context and the
// module with it; the next context gets a new id, so the address is resolved again.
// 0 when the id cannot be read (the address is then kept for the process).
unsigned long long current_ctx_id()
{
    typedef CUresult (*get_current_t)(CUcontext *);
    typedef CUresult (*get_id_t)(CUcontext, unsigned long long *);
    static get_current_t get_current = nullptr;
    static get_id_t get_id = nullptr;
    static bool looked = false;
    if (!looked) {
        looked = true;
        void *f1 = nullptr, *f2 = nullptr;
        cudaDriverEntryPointQueryResult q1, q2;
        if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &f1, 12000, cudaEnableDefault, &q1) == cudaSuccess &&
            q1 == cudaDriverEntryPointSuccess &&
            cudaGetDriverEntryPointByVersion("cuCtxGetId", &f2, 12000, cudaEnableDefault, &q2) == cudaSuccess &&
            q2 == cudaDriverEntryPointSuccess) {
            get_current = reinterpret_cast<get_current_t>(f1);
            get_id = reinterpret_cast<get_id_t>(f2);
        }
        cudaGetLastError();
    }
    CUcontext c = nullptr;
    unsigned long long id = 0;
    if (!get_current || !get_id || get_current(&c) != CUDA_SUCCESS || !c || get_id(c, &id) != CUDA_SUCCESS) return 0;
    return id;
}

sieve_status fail(const char *what, cudaError_t e)
{
    std::snprintf(gbs::g_last_cuda_error, sizeof gbs::g_last_cuda_error, "sieve_count_noalloc: %s: %s", what,
                  cudaGetErrorString(e));
    return SIEVE_ECUDA;
}

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
    // an error left pending by earlier work on this thread is reported as such and
    // left in place for its owner (nothing is launched)
    const cudaError_t pending = cudaPeekAtLastError();
    if (pending != cudaSuccess) return fail("error pending before the call (not cleared)", pending);
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return fail("cudaGetDevice", e);
    if (dev < 0 || dev >= kMaxDevices) return fail("device ordinal beyond the address table", cudaErrorInvalidDevice);
    unsigned long long *part;
    {
        // set-up, once per device (and again after a device reset), with that device current
        std::lock_guard<std::mutex> g(g_mu);
        const unsigned long long id = current_ctx_id();
        if (!g_addr[dev] || g_ctx_id[dev] != id) {
            void *p = nullptr;
            e = cudaGetSymbolAddress(&p, g_partials);
            if (e != cudaSuccess || !p) {
                cudaGetLastError();  // the failure is this call's own: consumed and reported
                return fail("cudaGetSymbolAddress(g_partials)", e != cudaSuccess ? e : cudaErrorInvalidSymbol);
            }
            g_addr[dev] = static_cast<unsigned long long *>(p);
            g_ctx_id[dev] = id;
        }
        part = g_addr[dev];
    }
    const uint64_t nwords = nbits / 32;
    const uint32_t nblocks = (uint32_t)((nwords + kWordsPerBlock - 1) / kWordsPerBlock);
    cudaStream_t st = (cudaStream_t)stream;
    if (nblocks) {
        k_partials<<<nblocks, 256, 0, st>>>(dev_bits, nwords, part);
        if ((e = cudaGetLastError()) != cudaSuccess) return fail("launch of k_partials", e);
    }
    k_total<<<1, 1024, 0, st>>>(part, nblocks, (unsigned long long *)dev_count);
    if ((e = cudaGetLastError()) != cudaSuccess) return fail("launch of k_total", e);
    return SIEVE_OK;
}
