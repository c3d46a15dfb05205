// fkmc_check.cu -- invariant check of one replica's device state.
//
// The fragment kMC conserves the number of vacancies and of H- ions (every
// event exchanges a vacancy with a neighbouring ion, Sec. II.A of
// arXiv:2004.09081), and the vacancy records that drive the fragment BKL must
// describe the occupancy exactly: one record per vacancy site, each listed by
// the fragment that owns its site.  This kernel pair measures all of that on
// the device, without a copy of the lattice to the host:
//   - a census of the occupancy codes (O, H-, V, and the unused code 3), with
//     a hash sum of the vacancy sites' linear indices;
//   - a pass over the fragment lists: record count, records whose site does
//     not hold a vacancy, records listed by a fragment that does not own the
//     site, records outside the lattice, fragments whose count is out of
//     range, and hash sums of the record sites and of the record ids.
// Equal hash sums of the vacancy sites and of the record sites (with equal
// counts) show the two multisets are equal up to a 2^-64 collision chance;
// the id sum is compared with that of 0 .. n_vac-1 on the host.
#include <cuda_runtime.h>

#include <algorithm>

#include "fkmc_check.h"

namespace fkmc {
namespace {

// sums of every thread's partial values, added to out[k] once per warp
__device__ __forceinline__ void warp_flush(unsigned long long* out, unsigned long long v[CHECK_WORDS])
{
    const unsigned FULL = 0xffffffffu;
#pragma unroll
    for (int k = 0; k < CHECK_WORDS; ++k) {
#pragma unroll
        for (int off = 16; off; off >>= 1) v[k] += __shfl_xor_sync(FULL, v[k], off);
    }
    if ((threadIdx.x & 31) == 0) {
#pragma unroll
        for (int k = 0; k < CHECK_WORDS; ++k)
            if (v[k]) atomicAdd(out + k, v[k]);
    }
}

__global__ void k_check_occupancy(RepDesc D, const uint32_t* __restrict__ occ, unsigned long long* out)
{
    unsigned long long v[CHECK_WORDS] = {};
    const int64_t words = 3ll * D.L[2] * D.L[1] * D.row_words;
    for (int64_t w = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; w < words;
         w += (int64_t)gridDim.x * blockDim.x) {
        const uint32_t word = occ[D.occ_word_off + w];
        const int64_t grp = w / 3;                  // (row, 16-cell block), the types interleaved
        const int t = (int)(w - grp * 3);
        const int64_t row = grp / D.row_words;      // z L1 + y
        const int x0 = (int)(grp - row * D.row_words) * 16;
        const int64_t z = row / D.L[1], y = row - z * D.L[1];
        const int64_t lin0 = (((int64_t)t * D.L[2] + z) * D.L[1] + y) * D.L[0] + x0;  // linear site index of x0
        for (int j = 0; j < 16 && x0 + j < D.L[0]; ++j) {
            const int code = (int)((word >> (2 * j)) & 3u);
            v[CHK_SITES + code] += 1ull;
            if (code == SP_V) v[CHK_HASH_VAC] += check_mix64((uint64_t)(lin0 + j));
        }
    }
    warp_flush(out, v);
}

__global__ void k_check_records(RepDesc D, const uint32_t* __restrict__ occ, const VacRec* __restrict__ recs,
                                const int32_t* __restrict__ counts, int cap, unsigned long long* out)
{
    unsigned long long v[CHECK_WORDS] = {};
    const int64_t nfrag = (int64_t)D.nf[0] * D.nf[1] * D.nf[2];
    for (int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; k < nfrag * cap;
         k += (int64_t)gridDim.x * blockDim.x) {
        const int64_t f = k / cap;
        const int s = (int)(k - f * cap);
        const int64_t g = D.frag_base + f;
        const int c = counts[g];
        if (s == 0 && (c < 0 || c > cap)) v[CHK_BAD_COUNT] += 1ull;
        if (s >= c) continue;
        const VacRec r = recs[g * cap + s];
        int t, x, y, z;
        split_key(r.key, t, x, y, z);
        if (t > 2 || x >= D.L[0] || y >= D.L[1] || z >= D.L[2]) {
            v[CHK_BAD_SITE] += 1ull;
            continue;
        }
        v[CHK_RECORDS] += 1ull;
        const uint32_t word = occ[occ_word(D, t, x, y, z)];
        if (((word >> occ_shift(x)) & 3u) != (uint32_t)SP_V) v[CHK_NOT_VAC] += 1ull;
        const int64_t owner = ((int64_t)frag_of(z, D.base[2], D.rem[2]) * D.nf[1] + frag_of(y, D.base[1], D.rem[1])) *
                                  D.nf[0] +
                              frag_of(x, D.base[0], D.rem[0]);
        if (owner != f) v[CHK_WRONG_FRAG] += 1ull;
        const int64_t lin = (((int64_t)t * D.L[2] + z) * D.L[1] + y) * D.L[0] + x;
        v[CHK_HASH_REC] += check_mix64((uint64_t)lin);
        v[CHK_HASH_ID] += check_mix64((uint64_t)r.id);
    }
    warp_flush(out, v);
}

}  // namespace

cudaError_t launch_check(const RepDesc& D, const uint32_t* occ, const VacRec* recs, const int32_t* counts, int cap,
                         unsigned long long* out, cudaStream_t st)
{
    cudaError_t e = cudaMemsetAsync(out, 0, sizeof(unsigned long long) * CHECK_WORDS, st);
    if (e != cudaSuccess) return e;
    int dev = 0, sms = 0;
    e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (e != cudaSuccess) return e;
    const int threads = 256;
    const int64_t words = 3ll * D.L[2] * D.L[1] * D.row_words;
    const int64_t slots = (int64_t)D.nf[0] * D.nf[1] * D.nf[2] * cap;
    auto grid = [&](int64_t items) {  // grid-stride beyond 8 blocks per SM
        const int64_t b = (items + threads - 1) / threads;
        return (unsigned)std::max<int64_t>(1, std::min<int64_t>(b, 8ll * sms));
    };
    k_check_occupancy<<<grid(words), threads, 0, st>>>(D, occ, out);
    e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    k_check_records<<<grid(slots), threads, 0, st>>>(D, occ, recs, counts, cap, out);
    return cudaGetLastError();
}

}  // namespace fkmc
