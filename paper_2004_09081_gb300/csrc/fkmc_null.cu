// fkmc_null.cu -- the atom-based fragment kMC with null events of
// arXiv:2004.09081 Sec. II.B (Eqs. AtomP, TimeStepFrg), the atoms being the
// vacancies.  One step over every replica of the batch, four launches:
//
//   k_null_rates    R_I of every vacancy; R_tot = sum, R_max = max (exact u64)
//   k_null_propose  N_frg picks (keyed bijection of the vacancy ids: an
//                   alternating Feistel network with hash rounds); each
//                   takes event i with probability q_i / R_max or the null
//                   event, and claims the two sites of its exchange with an
//                   atomic minimum of (step tag, pick index)
//   k_null_apply    a pick that holds both its claims applies its exchange
//                   (an earlier non-null pick sharing a site wins); the
//                   updated exchanges are disjoint and commute.  The last
//                   block to finish advances every replica's clock,
//                   clock += -ln(r') / R_tot * N_updated (Eq. TimeStepFrg)
//
// Rates are the mixed form's fixed point with F_null = 63 - ceil(log2(8 N_V)),
// so every sum is an exact integer and no reduction order enters the result.
#include <cuda_runtime.h>

#include <cstring>

#include <algorithm>

#include "fkmc_device.cuh"
#include "fkmc_kernels.h"

namespace fkmc {

namespace {

// replica of a vacancy (by = 0) or of a pick (by = 1)
__device__ __forceinline__ int null_replica(const RepDesc* descs, int nrep, int64_t v, int by)
{
    int lo = 0, hi = nrep - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        const int64_t start = by == 0 ? descs[mid].vac_off : descs[mid].pick_off;
        if (start <= v) lo = mid; else hi = mid - 1;
    }
    return lo;
}

// MurmurHash3's 64-bit finaliser (Appleby): three xor-shifts by 33 around its
// two published odd multipliers.
__device__ __forceinline__ uint64_t fmix64(uint64_t h)
{
    h ^= h >> 33;
    h *= 0xff51afd7ed558ccdull;
    h ^= h >> 33;
    h *= 0xc4ceb9fe1a85ec53ull;
    h ^= h >> 33;
    return h;
}

// Pick p of a step: the image of p under an alternating Feistel bijection of
// [0, 2^m), m = max(2, ceil(log2 n)), high part m - m/2 bits, low part m/2,
// twelve rounds (high, low, high, ...) of x ^= fmix64(other ^ k_r), walked back
// into [0, n).  k[4j + i] = word i of the step's Philox block (step, j) under
// (seed, replica, PICK), j = 0, 1, 2.
constexpr int NULL_PICK_ROUNDS = 12;
struct PickKeys {
    uint64_t k[NULL_PICK_ROUNDS];
};

__device__ __forceinline__ PickKeys pick_keys(uint64_t step, uint64_t seed, uint32_t replica)
{
    PickKeys pk;
#pragma unroll
    for (int j = 0; j < NULL_PICK_ROUNDS / 4; ++j) {
        const U64x4 b = philox4x64(step, (uint64_t)j, 0, 0, seed, key_word(replica, PURPOSE_PICK));
#pragma unroll
        for (int i = 0; i < 4; ++i) pk.k[4 * j + i] = b.x[i];
    }
    return pk;
}

__device__ __forceinline__ uint64_t null_pick(uint64_t p, uint64_t n, const PickKeys& pk)
{
    int m = 2;
    while ((1ull << m) < n) ++m;
    const int bl = m / 2, bh = m - bl;
    const uint64_t ml = (1ull << bl) - 1ull, mh = (1ull << bh) - 1ull;
    uint64_t v = p;
    do {
        uint64_t hi = v >> bl, lo = v & ml;
#pragma unroll
        for (int r = 0; r < NULL_PICK_ROUNDS; r += 2) {
            hi ^= fmix64(lo ^ pk.k[r]) & mh;
            lo ^= fmix64(hi ^ pk.k[r + 1]) & ml;
        }
        v = (hi << bl) | lo;
    } while (v >= n);
    return v;
}

__device__ __forceinline__ int64_t lin(const RepDesc& D, int t, int x, int y, int z)
{
    return (((int64_t)t * D.L[2] + z) * D.L[1] + y) * D.L[0] + x;
}

// fixed-point rate of neighbour n of a vacancy at (t, x, y, z); 0 for a
// vacancy; the raised table for a hop touching a grain-boundary cell (gb)
// The neighbour table in global memory: threads of a warp index it with
// different site types, which a kernel-parameter (constant bank) table would
// serve one distinct entry at a time.
__device__ __align__(8) NbEntry g_nbn[3][8];

__device__ __forceinline__ NbEntry null_nb(int t, int n)
{
    const uint2 v = __ldg(reinterpret_cast<const uint2*>(&g_nbn[0][0]) + 8 * t + n);
    NbEntry e;
    memcpy(&e, &v, sizeof e);
    return e;
}

__device__ __forceinline__ uint64_t null_rate(const RepDesc& D, const uint32_t* occ, const uint8_t* gb, int t, int x,
                                              int y, int z, int n)
{
    const NbEntry nb = null_nb(t, n);
    const int jx = wrapc(x + nb.dc[0], D.L[0]);
    const int jy = wrapc(y + nb.dc[1], D.L[1]);
    const int jz = wrapc(z + nb.dc[2], D.L[2]);
    const uint32_t w = __ldcg(occ + occ_word(D, nb.t2, jx, jy, jz));
    const int code = (int)((w >> occ_shift(jx)) & 3u);
    if (code == SP_V) return 0ull;
    const int ty = code * 3 + nb.d[2] + 1;
    if (gb && (gb[cell_index(D, x, y, z)] | gb[cell_index(D, jx, jy, jz)])) return D.qng[ty];
    return D.qn[ty];
}

// step tag of step k of a call: later steps have smaller tags, so a claim left
// by an earlier step never beats a claim of the current one
__device__ __forceinline__ uint64_t claim_of(uint64_t k, int64_t p)
{
    return ((uint64_t)(0xFFFFFFFEu - (uint32_t)k) << 32) | (uint64_t)(uint32_t)p;
}

__global__ void k_null_gather(const RepDesc* __restrict__ descs, int nrep, const VacRec* recs, const int32_t* counts,
                              int64_t nfrag_total, int cap, VacRec* vac, uint32_t* status)
{
    const int64_t total = nfrag_total * cap;
    for (int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; k < total;
         k += (int64_t)gridDim.x * blockDim.x) {
        const int64_t g = k / cap;
        const int slot = (int)(k % cap);
        if (slot >= counts[g]) continue;
        int lo = 0, hi = nrep - 1;
        while (lo < hi) {
            const int mid = (lo + hi + 1) >> 1;
            if (descs[mid].frag_base <= g) lo = mid; else hi = mid - 1;
        }
        const RepDesc& D = descs[lo];
        const VacRec r = recs[g * cap + slot];
        if ((int64_t)r.id < D.null_nv) vac[D.vac_off + r.id] = r;
        else atomicOr(status, STATUS_OVERFLOW);  // ids are 0 .. N_V-1 in a consistent state
    }
}

__global__ void k_null_scatter(const RepDesc* __restrict__ descs, int nrep, int64_t total_vac, const VacRec* vac,
                               VacRec* recs, int32_t* counts, int cap, uint32_t* status)
{
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < total_vac;
         i += (int64_t)gridDim.x * blockDim.x) {
        const RepDesc& D = descs[null_replica(descs, nrep, i, 0)];
        const VacRec r = vac[i];
        int t, x, y, z;
        split_key(r.key, t, x, y, z);
        const int64_t g = D.frag_base + ((int64_t)frag_of(z, D.base[2], D.rem[2]) * D.nf[1] +
                                         frag_of(y, D.base[1], D.rem[1])) * D.nf[0] + frag_of(x, D.base[0], D.rem[0]);
        const int slot = atomicAdd(counts + g, 1);
        if (slot < cap) recs[g * cap + slot] = r;
        else atomicOr(status, STATUS_OVERFLOW);
    }
}

// acc[3 r + 0] = R_tot, acc[3 r + 1] = R_max, acc[3 r + 2] = N_updated
__global__ void __launch_bounds__(256) k_null_rates(const RepDesc* __restrict__ descs, int nrep, int64_t total_vac,
                                                    const VacRec* __restrict__ vac, const uint32_t* occ,
                                                    const uint8_t* __restrict__ gb, unsigned long long* acc,
                                                    unsigned long long* nctl)
{
    if (blockIdx.x == 0 && threadIdx.x == 0) {  // nothing else in this launch reads nctl
        nctl[1] = nctl[0];
        nctl[0] = nctl[0] + 1;
    }
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const bool valid = i < total_vac;
    const int r = valid ? null_replica(descs, nrep, i, 0) : -1;
    unsigned long long R = 0ull;
    if (valid) {
        const RepDesc& D = descs[r];
        int t, x, y, z;
        split_key(vac[i].key, t, x, y, z);
#pragma unroll
        for (int n = 0; n < 8; ++n) R += null_rate(D, occ, gb, t, x, y, z, n);
    }
    const int r0 = __shfl_sync(0xffffffffu, r, 0);
    if (__all_sync(0xffffffffu, valid && r == r0)) {  // one replica: reduce in the warp first
        unsigned long long s = R, m = R;
#pragma unroll
        for (int off = 16; off; off >>= 1) {
            s += __shfl_xor_sync(0xffffffffu, s, off);
            m = max(m, __shfl_xor_sync(0xffffffffu, m, off));
        }
        if ((threadIdx.x & 31) == 0) {
            atomicAdd(acc + 3 * r0, s);
            atomicMax(acc + 3 * r0 + 1, m);
        }
    } else if (valid) {
        atomicAdd(acc + 3 * r, R);
        atomicMax(acc + 3 * r + 1, R);
    }
}

__global__ void __launch_bounds__(256) k_null_propose(const RepDesc* __restrict__ descs, int nrep, int64_t total_picks,
                                                      const VacRec* __restrict__ vac, const uint32_t* occ,
                                                      const uint8_t* __restrict__ gb, const unsigned long long* acc,
                                                      NullProp* props,
                                                      unsigned long long* claims, double* nE,
                                                      const unsigned long long* nctl)
{
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= total_picks) return;
    const int r = null_replica(descs, nrep, i, 1);
    const RepDesc& D = descs[r];
    const int64_t p = i - D.pick_off;
    const uint64_t k = nctl[1];
    const uint64_t step = D.null_step + k;
    const PickKeys rk = pick_keys(step, D.seed, D.replica);
    const int64_t id = (int64_t)null_pick((uint64_t)p, (uint64_t)D.null_nv, rk);
    int t, x, y, z;
    split_key(vac[D.vac_off + id].key, t, x, y, z);
    const U64x4 blk = philox4x64(step, (uint64_t)p, 0, 0, D.seed, key_word(D.replica, PURPOSE_NULL));
    const unsigned long long target = __umul64hi(blk.x[0], acc[3 * r + 1]);
    unsigned long long q[8];
#pragma unroll
    for (int n = 0; n < 8; ++n) q[n] = null_rate(D, occ, gb, t, x, y, z, n);  // 8 independent loads
    unsigned long long P = 0ull;
    int sel = -1;
#pragma unroll
    for (int n = 0; n < 8; ++n) {
        P += q[n];
        if (sel < 0 && P > target) sel = n;
    }
    if (p == 0) {  // the step's clock variate, off the critical path of the last apply block
        const U64x4 tb = philox4x64(step, ~0ull, 0, 0, D.seed, key_word(D.replica, PURPOSE_NULL));
        nE[r] = neglog64(tb.x[0]);
    }
    NullProp pr;
    pr.v = id;
    pr.n = sel;
    pr.pad = 0;
    props[i] = pr;
    if (sel < 0) return;
    const NbEntry nb = null_nb(t, sel);
    const unsigned long long mine = claim_of(k, p);
    atomicMin(claims + D.site_off + lin(D, t, x, y, z), mine);
    atomicMin(claims + D.site_off +
                  lin(D, nb.t2, wrapc(x + nb.dc[0], D.L[0]), wrapc(y + nb.dc[1], D.L[1]), wrapc(z + nb.dc[2], D.L[2])),
              mine);
}

// clock of replica r after a step: + -ln(r') / R_tot * N_updated, in units of
// 1/k32max (E = -ln(r'), r' from Philox (step, 2^64-1), drawn by the propose
// pass); hop counter; accumulators cleared
__device__ __forceinline__ void null_time(const RepDesc& D, int r, unsigned long long* acc, double* theta,
                                          unsigned long long* stats, const double* nE)
{
    const unsigned long long Rtot = __ldcg(acc + 3 * r), n = __ldcg(acc + 3 * r + 2);
    if (Rtot > 0ull) {
        const double E = __ldcg(nE + r);
        const double dth = __dmul_rn(__dmul_rn(__ddiv_rn(E, __ull2double_rn(Rtot)), D.two_pow_Fn), __ull2double_rn(n));
        theta[r] = __dadd_rn(theta[r], dth);
    }
    stats[2 * r] += n;
    acc[3 * r] = acc[3 * r + 1] = acc[3 * r + 2] = 0ull;
}

// nctl[2] counts the blocks of this launch that have finished
__global__ void __launch_bounds__(256) k_null_apply(const RepDesc* __restrict__ descs, int nrep, int64_t total_picks,
                                                    VacRec* vac, uint32_t* occ,
                                                    const NullProp* __restrict__ props,
                                                    const unsigned long long* claims, int32_t* tracer,
                                                    unsigned long long* acc, double* theta,
                                                    unsigned long long* stats, const double* nE,
                                                    unsigned long long* nctl)
{
    __shared__ bool last;
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const uint64_t k = nctl[1];
    bool did = false;
    int r = -1;
    if (i < total_picks) {
        r = null_replica(descs, nrep, i, 1);
        const RepDesc& D = descs[r];
        const NullProp pr = props[i];
        if (pr.n >= 0) {
            const int64_t p = i - D.pick_off;
            VacRec& v = vac[D.vac_off + pr.v];
            int t, x, y, z;
            split_key(v.key, t, x, y, z);
            const NbEntry nb = null_nb(t, pr.n);
            const int jx = wrapc(x + nb.dc[0], D.L[0]);
            const int jy = wrapc(y + nb.dc[1], D.L[1]);
            const int jz = wrapc(z + nb.dc[2], D.L[2]);
            const int64_t s_lin = lin(D, t, x, y, z), j_lin = lin(D, nb.t2, jx, jy, jz);
            const unsigned long long mine = claim_of(k, p);
            if (claims[D.site_off + s_lin] == mine && claims[D.site_off + j_lin] == mine) {
                const uint32_t w = __ldcg(occ + occ_word(D, nb.t2, jx, jy, jz));
                const uint32_t ion = (w >> occ_shift(jx)) & 3u;
                atomicXor(occ + occ_word(D, t, x, y, z), ((uint32_t)SP_V ^ ion) << occ_shift(x));
                atomicXor(occ + occ_word(D, nb.t2, jx, jy, jz), (ion ^ (uint32_t)SP_V) << occ_shift(jx));
                v.d[0] += nb.d[0];
                v.d[1] += nb.d[1];
                v.d[2] += nb.d[2];
                v.key = make_key(nb.t2, jx, jy, jz);
                if (tracer) {
                    int32_t* ts = tracer + 3 * (D.site_off + s_lin);
                    int32_t* tj = tracer + 3 * (D.site_off + j_lin);
                    ts[0] = tj[0] - nb.d[0];
                    ts[1] = tj[1] - nb.d[1];
                    ts[2] = tj[2] - nb.d[2];
                    tj[0] = tj[1] = tj[2] = 0;
                }
                did = true;
            }
        }
    }
    const int r0 = __shfl_sync(0xffffffffu, r, 0);
    if (__all_sync(0xffffffffu, r == r0)) {
        const unsigned n = __popc(__ballot_sync(0xffffffffu, did));
        if ((threadIdx.x & 31) == 0 && n) atomicAdd(acc + 3 * r0 + 2, (unsigned long long)n);
    } else if (did) {
        atomicAdd(acc + 3 * r + 2, 1ull);
    }
    // the last block to finish closes the step (threadFenceReduction pattern)
    __threadfence();
    __syncthreads();
    if (threadIdx.x == 0) last = atomicAdd(nctl + 2, 1ull) == (unsigned long long)(gridDim.x - 1);
    __syncthreads();
    if (!last) return;
    __threadfence();
    for (int q = threadIdx.x; q < nrep; q += blockDim.x) null_time(descs[q], q, acc, theta, stats, nE);
    if (threadIdx.x == 0) nctl[2] = 0ull;
}

constexpr int NT = 256;

unsigned grid_of(int64_t n)
{
    return (unsigned)std::max<int64_t>(1, std::min<int64_t>((n + NT - 1) / NT, 1 << 30));
}

}  // namespace

cudaError_t launch_null_gather(const RepDesc* d_descs, int nrep, const VacRec* recs, const int32_t* counts,
                               int64_t nfrag_total, int cap, VacRec* vac, uint32_t* status, cudaStream_t st)
{
    const unsigned blocks = (unsigned)std::min<int64_t>(65536, std::max<int64_t>(1, (nfrag_total * cap + NT - 1) / NT));
    k_null_gather<<<blocks, NT, 0, st>>>(d_descs, nrep, recs, counts, nfrag_total, cap, vac, status);
    return cudaGetLastError();
}

cudaError_t launch_null_scatter(const RepDesc* d_descs, int nrep, int64_t total_vac, const VacRec* vac,
                                VacRec* recs, int32_t* counts, int64_t nfrag_total, int cap, uint32_t* status,
                                cudaStream_t st)
{
    cudaError_t e = cudaMemsetAsync(counts, 0, sizeof(int32_t) * nfrag_total, st);
    if (e != cudaSuccess || total_vac == 0) return e;
    const unsigned blocks = (unsigned)std::min<int64_t>(65536, (total_vac + NT - 1) / NT);
    k_null_scatter<<<blocks, NT, 0, st>>>(d_descs, nrep, total_vac, vac, recs, counts, cap, status);
    return cudaGetLastError();
}

cudaError_t null_upload_neighbours(const NbEntry* host24)
{
    return cudaMemcpyToSymbol(g_nbn, host24, sizeof(NbEntry) * 24);
}

// One step of every replica (three launches; fixed arguments, so a graph can
// hold it).  nctl[2] must be 0 before the first step.
cudaError_t launch_null_step(const RepDesc* d_descs, int nrep, int64_t total_vac, int64_t total_picks, VacRec* vac,
                             uint32_t* occ, const uint8_t* gb, unsigned long long* acc,
                             NullProp* props,
                             unsigned long long* claims, int32_t* tracer, double* theta, double* nE,
                             unsigned long long* stats, unsigned long long* nctl, cudaStream_t st)
{
    k_null_rates<<<grid_of(total_vac), NT, 0, st>>>(d_descs, nrep, total_vac, vac, occ, gb, acc, nctl);
    k_null_propose<<<grid_of(total_picks), NT, 0, st>>>(d_descs, nrep, total_picks, vac, occ, gb, acc, props,
                                                        claims, nE, nctl);
    k_null_apply<<<grid_of(total_picks), NT, 0, st>>>(d_descs, nrep, total_picks, vac, occ, props, claims, tracer,
                                                      acc, theta, stats, nE, nctl);
    return cudaGetLastError();
}

}  // namespace fkmc
