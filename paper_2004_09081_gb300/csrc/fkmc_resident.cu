// fkmc_resident.cu -- replica-resident window kernel (mixed form).
//
// One CTA owns one replica for a whole kmc_run call: the replica's packed
// occupancy is staged into shared memory with TMA bulk copies
// (cp.async.bulk + mbarrier), its vacancy records are unpacked into
// shared-memory arrays linked per fragment, and the CTA runs every window and
// colour phase with __syncthreads() between phases -- no grid-wide
// synchronisation, because replicas are independent.  Inside a phase one
// thread runs one fragment's BKL (arXiv:2004.09081 Sec. II.A Eqs.
// RateCnst1, eventSelection, TimeStep; fragment-local selection Sec. II.B
// Eq. AtomP).  Selection uses exact u64 fixed-point sums, so the result is
// identical to the warp kernel and to the oracle's mixed form.  At the end the
// occupancy goes back to global memory with a TMA bulk store and the records
// go back to the per-fragment lists.
#include <cuda_runtime.h>

#include "fkmc_device.cuh"
#include "fkmc_kernels.h"

namespace fkmc {

namespace {

__device__ __forceinline__ uint32_t smem_u32(const void* p)
{
    return (uint32_t)__cvta_generic_to_shared(p);
}

__device__ __forceinline__ uint64_t globaltimer()
{
    uint64_t t;
    asm volatile("mov.u64 %0, %globaltimer;" : "=l"(t));
    return t;
}

__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t* bar, uint32_t bytes)
{
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes)
                 : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, uint32_t parity)
{
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(smem_u32(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}

// Bounded wait: gives up after `ns` nanoseconds and reports it.
__device__ __forceinline__ bool mbar_wait_bounded(uint64_t* bar, uint32_t parity, uint64_t ns)
{
    const uint64_t t0 = globaltimer();
    while (!mbar_try_wait(bar, parity))
        if (globaltimer() - t0 > ns) return false;
    return true;
}

__device__ __forceinline__ void bulk_g2s(void* dst, const void* src, uint32_t bytes, uint64_t* bar)
{
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
            smem_u32(dst)),
        "l"(src), "r"(bytes), "r"(smem_u32(bar))
        : "memory");
}

__device__ __forceinline__ void bulk_s2g(void* dst, const void* src, uint32_t bytes)
{
    asm volatile("cp.async.bulk.global.shared::cta.bulk_group [%0], [%1], %2;" ::"l"(dst), "r"(smem_u32(src)),
                 "r"(bytes)
                 : "memory");
}

constexpr uint32_t BULK_CHUNK = 32768;  // bytes per bulk copy instruction
constexpr uint64_t WAIT_NS = 2000000000ull;  // 2 s bound on any device-side wait

struct Shared {
    RepDesc D;
    NbEntry nb[3][8];
    uint64_t bar;
    int perm[8];
    int nv_count;
    unsigned long long hops, hand;
    int abort;
};

}  // namespace

size_t resident_smem_bytes(const RepDesc& D, int64_t n_vac)
{
    const int64_t words = 3 * (int64_t)D.L[2] * D.L[1] * D.row_words;
    const int64_t nfrag = (int64_t)D.nf[0] * D.nf[1] * D.nf[2];
    size_t b = (size_t)words * 4;                 // occupancy
    b += (size_t)n_vac * (8 + 12 + 4 + 4);        // key, d[3], id, next
    b += (size_t)nfrag * 4;                       // list heads
    return (b + 127) & ~(size_t)127;
}

__global__ void __launch_bounds__(256) k_resident(const RepDesc* __restrict__ descs,
                                                  const int32_t* __restrict__ reps,
                                                  const int64_t* __restrict__ nvac, uint64_t windows,
                                                  uint32_t* occ, VacRec* recs, int32_t* counts,
                                                  int32_t* tracer, unsigned long long* stats,
                                                  uint32_t* status, int cap, NbTable nbt)
{
    extern __shared__ __align__(128) unsigned char dyn[];
    __shared__ Shared sh;
    const int tid = threadIdx.x;
    const int r = reps[blockIdx.x];
    const int64_t n_vac = nvac[r];

    if (tid == 0) {
        sh.D = descs[r];
        sh.nv_count = 0;
        sh.hops = 0;
        sh.hand = 0;
        sh.abort = 0;
    }
    if (tid < 24) (&sh.nb[0][0])[tid] = (&nbt.e[0][0])[tid];  // threads index it with different t
    __syncthreads();
    const RepDesc& D = sh.D;
    const int64_t words = 3 * (int64_t)D.L[2] * D.L[1] * D.row_words;
    const int64_t nfrag = (int64_t)D.nf[0] * D.nf[1] * D.nf[2];
    uint32_t* occ_s = reinterpret_cast<uint32_t*>(dyn);
    uint64_t* key_s = reinterpret_cast<uint64_t*>(dyn + ((words * 4 + 15) & ~15ll));
    int32_t* d_s = reinterpret_cast<int32_t*>(key_s + n_vac);
    uint32_t* id_s = reinterpret_cast<uint32_t*>(d_s + 3 * n_vac);
    int32_t* next_s = reinterpret_cast<int32_t*>(id_s + n_vac);
    int32_t* head_s = next_s + n_vac;

    // ---- stage in: occupancy by TMA bulk copies, records by plain loads
    const uint32_t occ_bytes = (uint32_t)(words * 4);
    if (tid == 0) {
        mbar_init(&sh.bar, 1);
        mbar_arrive_expect_tx(&sh.bar, occ_bytes);
        const char* src = reinterpret_cast<const char*>(occ + D.occ_word_off);
        for (uint32_t off = 0; off < occ_bytes; off += BULK_CHUNK) {
            const uint32_t n = min(BULK_CHUNK, occ_bytes - off);
            bulk_g2s(dyn + off, src + off, n, &sh.bar);
        }
    }
    for (int64_t f = tid; f < nfrag; f += blockDim.x) {
        const int64_t g = D.frag_base + f;
        const int c = counts[g];
        int head = -1;
        for (int k = 0; k < c && k < cap; ++k) {
            const int v = atomicAdd(&sh.nv_count, 1);
            if (v >= n_vac) {
                atomicOr(status, STATUS_OVERFLOW);
                break;
            }
            const VacRec rr = recs[g * cap + k];
            key_s[v] = rr.key;
            d_s[3 * v] = rr.d[0];
            d_s[3 * v + 1] = rr.d[1];
            d_s[3 * v + 2] = rr.d[2];
            id_s[v] = rr.id;
            next_s[v] = head;
            head = v;
        }
        if (c > cap) atomicOr(status, STATUS_OVERFLOW);
        head_s[f] = head;
    }
    __syncthreads();  // the barrier init is visible to every thread from here on
    if (!mbar_wait_bounded(&sh.bar, 0, WAIT_NS)) {
        if (tid == 0) {
            atomicOr(status, STATUS_TIMEOUT);
            sh.abort = 1;
        }
        mbar_wait_bounded(&sh.bar, 0, WAIT_NS);  // let copies in flight land before leaving
    }
    __syncthreads();
    if (sh.abort) return;

    const uint64_t hop_k1 = key_word(D.replica, PURPOSE_HOP);
    unsigned long long my_hops = 0, my_hand = 0;
    uint16_t sl[RESIDENT_MAX_SLOTS];  // slot -> vacancy index (bit 15: slot dead)

    for (uint64_t wk = 0; wk < windows; ++wk) {
        const uint64_t w = D.window + wk;
        if (tid < 32) {
            const int c = colour_of_phase(D.seed, D.replica, w, tid & 7, tid);
            if (tid < 8) sh.perm[tid] = c;
        }
        __syncthreads();
        for (int p = 0; p < 8; ++p) {
            const int colour = sh.perm[p];
            int cnt[3], bit[3];
#pragma unroll
            for (int d = 0; d < 3; ++d) {
                bit[d] = (colour >> d) & 1;
                cnt[d] = D.nf[d] == 1 ? (bit[d] == 0 ? 1 : 0) : D.nf[d] / 2;
            }
            const int ncls = cnt[0] * cnt[1] * cnt[2];
            for (int l = tid; l < ncls; l += blockDim.x) {
                int f[3], lo_c[3], hi_c[3];
                f[0] = l % cnt[0];
                f[1] = (l / cnt[0]) % cnt[1];
                f[2] = l / (cnt[0] * cnt[1]);
#pragma unroll
                for (int d = 0; d < 3; ++d) {
                    f[d] = D.nf[d] == 1 ? 0 : 2 * f[d] + bit[d];
                    lo_c[d] = frag_start(f[d], D.base[d], D.rem[d]);
                    hi_c[d] = frag_start(f[d] + 1, D.base[d], D.rem[d]);
                }
                const int fid = (f[2] * D.nf[1] + f[1]) * D.nf[0] + f[0];
                // slots: the fragment's vacancies in ascending site order
                int n = 0;
                for (int v = head_s[fid]; v >= 0; v = next_s[v]) {
                    if (n >= cap || n >= RESIDENT_MAX_SLOTS) {
                        atomicOr(status, STATUS_OVERFLOW);
                        break;
                    }
                    const uint64_t k = key_s[v];
                    int m = n++;
                    while (m > 0 && key_s[sl[m - 1]] > k) {
                        sl[m] = sl[m - 1];
                        --m;
                    }
                    sl[m] = (uint16_t)v;
                }
                if (n == 0) continue;

                double clock = 0.0;
                uint64_t i = 0, blk_id = ~0ull;
                U64x4 blk;
                blk.x[0] = blk.x[1] = blk.x[2] = blk.x[3] = 0;
                for (;;) {
                    // exact fixed-point total of the fragment's events
                    unsigned long long S = 0;
                    for (int m = 0; m < n; ++m) {
                        if (sl[m] & 0x8000u) continue;
                        int t, x, y, z;
                        split_key(key_s[sl[m]], t, x, y, z);
#pragma unroll
                        for (int q = 0; q < 8; ++q) {
                            const NbEntry nb = sh.nb[t][q];
                            const int jx = wrapc(x + nb.dc[0], D.L[0]);
                            const int jy = wrapc(y + nb.dc[1], D.L[1]);
                            const int jz = wrapc(z + nb.dc[2], D.L[2]);
                            const uint32_t wd =
                                occ_s[(((int64_t)nb.t2 * D.L[2] + jz) * D.L[1] + jy) * D.row_words + (jx >> 4)];
                            const int code = (int)((wd >> occ_shift(jx)) & 3u);
                            if (code != SP_V) S += D.q[code * 3 + nb.d[2] + 1];
                        }
                    }
                    if (S == 0) break;
                    if (i >= MAX_EVENTS_PER_PHASE) {
                        atomicOr(status, STATUS_EVENT_LIMIT);
                        break;
                    }
                    if ((i >> 1) != blk_id) {
                        blk_id = i >> 1;
                        blk = philox4x64((uint64_t)fid, w, blk_id, 0, D.seed, hop_k1);
                    }
                    const uint64_t xt = (i & 1) ? blk.x[2] : blk.x[0];
                    const uint64_t xs = (i & 1) ? blk.x[3] : blk.x[1];
                    const float E = neglog32(xt);
                    const float ratio = __fdiv_rn(E, __ull2float_rn(S));
                    const double dth = __dmul_rn((double)ratio, D.two_pow_F);
                    if (__dadd_rn(clock, dth) > D.theta_tau) break;
                    const unsigned long long target = __umul64hi(xs, S);
                    // first event whose running sum exceeds the target
                    unsigned long long P = 0;
                    int sm_ = -1, sq = -1, ion = 0;
                    for (int m = 0; m < n && sm_ < 0; ++m) {
                        if (sl[m] & 0x8000u) continue;
                        int t, x, y, z;
                        split_key(key_s[sl[m]], t, x, y, z);
                        for (int q = 0; q < 8; ++q) {
                            const NbEntry nb = sh.nb[t][q];
                            const int jx = wrapc(x + nb.dc[0], D.L[0]);
                            const int jy = wrapc(y + nb.dc[1], D.L[1]);
                            const int jz = wrapc(z + nb.dc[2], D.L[2]);
                            const uint32_t wd =
                                occ_s[(((int64_t)nb.t2 * D.L[2] + jz) * D.L[1] + jy) * D.row_words + (jx >> 4)];
                            const int code = (int)((wd >> occ_shift(jx)) & 3u);
                            if (code == SP_V) continue;
                            P += D.q[code * 3 + nb.d[2] + 1];
                            if (P > target) {
                                sm_ = m;
                                sq = q;
                                ion = code;
                                break;
                            }
                        }
                    }
                    // apply the exchange
                    const int v = sl[sm_];
                    int t, x, y, z;
                    split_key(key_s[v], t, x, y, z);
                    const NbEntry nb = sh.nb[t][sq];
                    const int jx = wrapc(x + nb.dc[0], D.L[0]);
                    const int jy = wrapc(y + nb.dc[1], D.L[1]);
                    const int jz = wrapc(z + nb.dc[2], D.L[2]);
                    atomicXor(occ_s + (((int64_t)t * D.L[2] + z) * D.L[1] + y) * D.row_words + (x >> 4),
                              ((uint32_t)SP_V ^ (uint32_t)ion) << occ_shift(x));
                    atomicXor(occ_s + (((int64_t)nb.t2 * D.L[2] + jz) * D.L[1] + jy) * D.row_words + (jx >> 4),
                              ((uint32_t)ion ^ (uint32_t)SP_V) << occ_shift(jx));
                    d_s[3 * v] += nb.d[0];
                    d_s[3 * v + 1] += nb.d[1];
                    d_s[3 * v + 2] += nb.d[2];
                    if (tracer) {
                        const int64_t s_lin = (((int64_t)t * D.L[2] + z) * D.L[1] + y) * D.L[0] + x;
                        const int64_t j_lin = (((int64_t)nb.t2 * D.L[2] + jz) * D.L[1] + jy) * D.L[0] + jx;
                        int32_t* ts = tracer + 3 * (D.site_off + s_lin);
                        int32_t* tj = tracer + 3 * (D.site_off + j_lin);
                        ts[0] = tj[0] - nb.d[0];
                        ts[1] = tj[1] - nb.d[1];
                        ts[2] = tj[2] - nb.d[2];
                        tj[0] = tj[1] = tj[2] = 0;
                    }
                    key_s[v] = make_key(nb.t2, jx, jy, jz);
                    const bool owned = jx >= lo_c[0] && jx < hi_c[0] && jy >= lo_c[1] && jy < hi_c[1] &&
                                       jz >= lo_c[2] && jz < hi_c[2];
                    if (!owned) {
                        const int gx = frag_of(jx, D.base[0], D.rem[0]);
                        const int gy = frag_of(jy, D.base[1], D.rem[1]);
                        const int gz = frag_of(jz, D.base[2], D.rem[2]);
                        const int g2 = (gz * D.nf[1] + gy) * D.nf[0] + gx;
                        next_s[v] = atomicExch(head_s + g2, v);
                        sl[sm_] |= 0x8000u;
                        ++my_hand;
                    }
                    clock = __dadd_rn(clock, dth);
                    ++i;
                }
                my_hops += i;
                // surviving vacancies stay linked to this fragment
                int head = -1;
                for (int m = 0; m < n; ++m) {
                    if (sl[m] & 0x8000u) continue;
                    next_s[sl[m]] = head;
                    head = sl[m];
                }
                head_s[fid] = head;
            }
            __syncthreads();
        }
    }

    // ---- stage out: occupancy by a TMA bulk store, records to the fragment lists
    if (tid == 0) {
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        char* dst = reinterpret_cast<char*>(occ + D.occ_word_off);
        for (uint32_t off = 0; off < occ_bytes; off += BULK_CHUNK) {
            const uint32_t nb = min(BULK_CHUNK, occ_bytes - off);
            bulk_s2g(dst + off, dyn + off, nb);
        }
        asm volatile("cp.async.bulk.commit_group;" ::: "memory");
    }
    for (int64_t f = tid; f < nfrag; f += blockDim.x) {
        const int64_t g = D.frag_base + f;
        int k = 0;
        for (int v = head_s[f]; v >= 0; v = next_s[v], ++k) {
            if (k >= cap) {
                atomicOr(status, STATUS_OVERFLOW);
                break;
            }
            VacRec rr;
            rr.key = key_s[v];
            rr.d[0] = d_s[3 * v];
            rr.d[1] = d_s[3 * v + 1];
            rr.d[2] = d_s[3 * v + 2];
            rr.id = id_s[v];
            recs[g * cap + k] = rr;
        }
        counts[g] = k;
    }
    atomicAdd(&sh.hops, my_hops);
    atomicAdd(&sh.hand, my_hand);
    __syncthreads();
    if (tid == 0) {
        if (sh.hops) atomicAdd(stats + 2 * r, sh.hops);
        if (sh.hand) atomicAdd(stats + 2 * r + 1, sh.hand);
        asm volatile("cp.async.bulk.wait_group 0;" ::: "memory");
    }
}

cudaError_t resident_prepare()
{
    return cudaFuncSetAttribute(k_resident, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                (int)RESIDENT_MAX_SMEM);
}

cudaError_t launch_resident(const RepDesc* d_descs, const int32_t* d_reps, int nreps, const int64_t* d_nvac,
                            size_t smem, uint64_t windows, uint32_t* occ, VacRec* recs, int32_t* counts,
                            int32_t* tracer, unsigned long long* stats, uint32_t* status, int cap,
                            const NbTable& nbt, cudaStream_t st)
{
    if (nreps <= 0) return cudaSuccess;
    k_resident<<<nreps, 256, smem, st>>>(d_descs, d_reps, d_nvac, windows, occ, recs, counts, tracer, stats,
                                         status, cap, nbt);
    return cudaGetLastError();
}

}  // namespace fkmc
