// fkmc_check.h -- the invariant check of one replica's state (fkmc_check.cu).
#pragma once
#include <cuda_runtime.h>

#include <cstdint>

#include "fkmc_device.cuh"

namespace fkmc {

// invariant check of one replica's state (fkmc_check.cu): out[CHECK_WORDS] gets
// the occupancy census (CHK_SITES + code, code 3 unused), the record count and
// the counts of records not on a vacancy, in the wrong fragment or outside the
// lattice, of fragments with a count outside [0, cap], and hash sums of the
// vacancy sites, the record sites and the record ids (mod 2^64)
constexpr int CHK_SITES = 0, CHK_RECORDS = 4, CHK_NOT_VAC = 5, CHK_WRONG_FRAG = 6, CHK_BAD_SITE = 7,
              CHK_BAD_COUNT = 8, CHK_HASH_VAC = 9, CHK_HASH_REC = 10, CHK_HASH_ID = 11, CHECK_WORDS = 12;
// SplitMix64's output step (Steele, Lea and Flood, OOPSLA 2014): the Weyl
// increment, then the xor-shift-multiply finaliser with Stafford's "Mix13"
// constants; a bijection of the 64-bit words with no fixed point at 0
__host__ __device__ inline uint64_t check_mix64(uint64_t z)
{
    z += 0x9e3779b97f4a7c15ull;
    z = (z ^ (z >> 30)) * 0xbf58476d1ce4e5b9ull;
    z = (z ^ (z >> 27)) * 0x94d049bb133111ebull;
    return z ^ (z >> 31);
}
cudaError_t launch_check(const RepDesc& D, const uint32_t* occ, const VacRec* recs, const int32_t* counts, int cap,
                         unsigned long long* out, cudaStream_t st);

}  // namespace fkmc
