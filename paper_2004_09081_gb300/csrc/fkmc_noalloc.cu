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

__global__ void k_moments_groups(const VacRec* __restrict__ recs, const int32_t* __restrict__ counts,
                                 int n_groups, int cap, NoAllocScratch* s)
{
    const long long nfrag = s->off[n_groups];
    const long long total = nfrag * cap;
    for (long long k = (long long)blockIdx.x * blockDim.x + threadIdx.x; k < total;
         k += (long long)gridDim.x * blockDim.x) {
        const long long f = k / cap;
        const int slot = (int)(k % cap);
        if (slot >= counts[f]) continue;
        int lo = 0, hi = n_groups - 1;
        while (lo < hi) {
            const int mid = (lo + hi + 1) >> 1;
            if (s->off[mid] <= f) lo = mid; else hi = mid - 1;
        }
        const VacRec r = recs[f * cap + slot];
        unsigned long long* o = s->acc + 7 * lo;
        atomicAdd(o, 1ull);
#pragma unroll
        for (int d = 0; d < 3; ++d) {
            if (r.d[d]) {
                atomicAdd(o + 1 + d, (unsigned long long)(long long)r.d[d]);
                atomicAdd(o + 4 + d, (unsigned long long)((long long)r.d[d] * r.d[d]));
            }
        }
    }
}

constexpr int MAX_DEVICES = 64;
std::mutex g_setup_mutex;
NoAllocScratch* g_scratch_ptr[MAX_DEVICES] = {};

// Device address of the scratch on the current device, looked up once per device.
int scratch_for_current_device(NoAllocScratch** out)
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
        g_scratch_ptr[dev] = static_cast<NoAllocScratch*>(p);
    }
    *out = g_scratch_ptr[dev];
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
    NoAllocScratch* s = nullptr;
    int rc = scratch_for_current_device(&s);
    if (rc) return rc;
    cudaStream_t st = (cudaStream_t)stream;
    const long long nfrag = fragment_offsets[n_groups];
    cudaError_t e = cudaMemcpyAsync(s->off, fragment_offsets, sizeof(long long) * (n_groups + 1),
                                    cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess) e = cudaMemsetAsync(s->acc, 0, sizeof(unsigned long long) * 7 * n_groups, st);
    if (e == cudaSuccess && nfrag > 0) {
        const int threads = 256;
        long long blocks = (nfrag * cap_v + threads - 1) / threads;
        if (blocks > 8 * 152) blocks = 8 * 152;
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
