// fkmc_noalloc.cu -- vacancy-moment reduction that allocates nothing.
//
// Same reduction as kmc_read_moments_all (exact integer moments of the
// vacancy displacements, grouped per replica), but over device buffers the
// caller owns and with its only scratch -- the group offsets and the
// accumulators -- in a file-scope static device array.  It serves callers
// that cannot allocate device memory: a host framework that owns every
// device allocation through its own pool, a plugin that is handed fixed
// buffers, or a serving loop whose memory is planned ahead and may not grow.
#include <cuda_runtime.h>

#include <cstdint>
#include <cstring>
#include <mutex>

#include "fkmc.h"
#include "fkmc_device.cuh"
#include "fkmc_kernels.h"

namespace fkmc {
namespace {

struct NoAllocScratch {
    long long off[FKMC_NOALLOC_MAX_GROUPS + 1];           // fragment offset of each group
    unsigned long long acc[7 * FKMC_NOALLOC_MAX_GROUPS];  // moments of each group
};

// Held by every GPU that loads the library, until the process exits.  In host
// code this name is only a stand-in: its device address comes from
// cudaGetSymbolAddress, once per device.
static __device__ __align__(256) NoAllocScratch g_noalloc_scratch;

__device__ __forceinline__ void flush_group(NoAllocScratch* s, int g, const unsigned long long acc[7])
{
    if (g < 0 || acc[0] == 0ull) return;
    unsigned long long* o = s->acc + 7 * g;
#pragma unroll
    for (int k = 0; k < 7; ++k)
        if (acc[k]) atomicAdd(o + k, acc[k]);
}

// Groups own contiguous fragment ranges and a thread's slots k ascend, so its
// group index only grows: it sums its records in registers and adds them to
// the group's accumulators when the group changes and at the end, where the
// lanes of a warp that end in the same group first combine by shuffles.
__global__ void k_moments_groups(const VacRec* __restrict__ recs, const int32_t* __restrict__ counts,
                                 int n_groups, int cap, NoAllocScratch* s)
{
    const long long nfrag = s->off[n_groups];
    const long long total = nfrag * cap;
    unsigned long long acc[7] = {0ull, 0ull, 0ull, 0ull, 0ull, 0ull, 0ull};
    int cur = -1;
    for (long long k = (long long)blockIdx.x * blockDim.x + threadIdx.x; k < total;
         k += (long long)gridDim.x * blockDim.x) {
        const long long f = k / cap;
        const int slot = (int)(k % cap);
        if (slot >= counts[f]) continue;
        int lo = 0, hi = n_groups - 1;  // the last group whose first fragment is <= f
        while (lo < hi) {
            const int mid = (lo + hi + 1) >> 1;
            if (s->off[mid] <= f) lo = mid; else hi = mid - 1;
        }
        if (lo != cur) {
            flush_group(s, cur, acc);
#pragma unroll
            for (int q = 0; q < 7; ++q) acc[q] = 0ull;
            cur = lo;
        }
        const VacRec r = recs[f * cap + slot];
        acc[0] += 1ull;
#pragma unroll
        for (int d = 0; d < 3; ++d) {
            acc[1 + d] += (unsigned long long)(long long)r.d[d];
            acc[4 + d] += (unsigned long long)((long long)r.d[d] * r.d[d]);
        }
    }
    const unsigned FULL = 0xffffffffu;
    const int lead = __shfl_sync(FULL, cur, 0);
    if (__all_sync(FULL, cur == lead)) {
#pragma unroll
        for (int q = 0; q < 7; ++q)
#pragma unroll
            for (int off = 16; off; off >>= 1) acc[q] += __shfl_xor_sync(FULL, acc[q], off);
        if ((threadIdx.x & 31) == 0) flush_group(s, cur, acc);
    } else {
        flush_group(s, cur, acc);
    }
}

constexpr int MAX_DEVICES = 64;
std::mutex g_setup_mutex;
NoAllocScratch* g_scratch_ptr[MAX_DEVICES] = {};
int g_sm_count[MAX_DEVICES] = {};

// Device address of the scratch on the current device and its SM count,
// looked up once per device.
int scratch_for_current_device(NoAllocScratch** out, int* sms)
{
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return set_error(FKMC_ECUDA, cudaGetErrorString(e));
    if (dev < 0 || dev >= MAX_DEVICES) return set_error(FKMC_EINVAL, "device index beyond 63");
    std::lock_guard<std::mutex> lock(g_setup_mutex);
    if (!g_scratch_ptr[dev]) {
        void* p = nullptr;
        e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess || !p)
            return set_error(FKMC_ECUDA, e != cudaSuccess ? cudaGetErrorString(e) : "null symbol address");
        int n = 0;
        e = cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev);
        if (e != cudaSuccess || n < 1)
            return set_error(FKMC_ECUDA, e != cudaSuccess ? cudaGetErrorString(e) : "no multiprocessors");
        g_sm_count[dev] = n;
        g_scratch_ptr[dev] = static_cast<NoAllocScratch*>(p);
    }
    *out = g_scratch_ptr[dev];
    *sms = g_sm_count[dev];
    return FKMC_OK;
}

}  // namespace
}  // namespace fkmc

using namespace fkmc;

extern "C" int kmc_vacancy_moments_noalloc(const void* d_records, const int32_t* d_counts,
                                           const int64_t* fragment_offsets, int32_t n_groups, int32_t cap_v,
                                           int64_t* out, void* stream)
{
    if (!d_records || !d_counts || !fragment_offsets || !out)
        return set_error(FKMC_EINVAL, "null pointer argument");
    if (n_groups < 1 || n_groups > FKMC_NOALLOC_MAX_GROUPS)
        return set_error(FKMC_EINVAL, "n_groups must be in [1, FKMC_NOALLOC_MAX_GROUPS = 4096]");
    if (cap_v < 1 || cap_v > 256) return set_error(FKMC_EINVAL, "cap_v must be in [1, 256]");
    if (fragment_offsets[0] != 0) return set_error(FKMC_EINVAL, "fragment_offsets[0] must be 0");
    for (int g = 0; g < n_groups; ++g)
        if (fragment_offsets[g + 1] < fragment_offsets[g])
            return set_error(FKMC_EINVAL, "fragment_offsets must not decrease");
    const long long nfrag = fragment_offsets[n_groups];
    if (nfrag > INT64_MAX / cap_v) return set_error(FKMC_EINVAL, "fragment_offsets[n_groups] x cap_v overflows");
    cudaStream_t st = (cudaStream_t)stream;
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    cudaError_t e = cudaStreamIsCapturing(st, &cs);
    if (e != cudaSuccess) return set_error(FKMC_ECUDA, cudaGetErrorString(e));
    if (cs != cudaStreamCaptureStatusNone)
        return set_error(FKMC_EINVAL, "the call is synchronous: its stream must not be capturing");
    NoAllocScratch* s = nullptr;
    int sms = 0;
    int rc = scratch_for_current_device(&s, &sms);
    if (rc) return rc;
    e = cudaMemcpyAsync(s->off, fragment_offsets, sizeof(long long) * (n_groups + 1), cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess) e = cudaMemsetAsync(s->acc, 0, sizeof(unsigned long long) * 7 * n_groups, st);
    if (e == cudaSuccess && nfrag > 0) {
        const int threads = 256;
        long long blocks = (nfrag * cap_v + threads - 1) / threads;
        if (blocks > 8ll * sms) blocks = 8ll * sms;  // grid-stride beyond that
        k_moments_groups<<<(unsigned)blocks, threads, 0, st>>>(static_cast<const VacRec*>(d_records), d_counts,
                                                               n_groups, cap_v, s);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(out, s->acc, sizeof(int64_t) * 7 * n_groups, cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) return set_error(FKMC_ECUDA, cudaGetErrorString(e));
    return FKMC_OK;
}
