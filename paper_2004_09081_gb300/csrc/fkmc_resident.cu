// fkmc_resident.cu -- replica-resident window kernel (mixed form).
//
// One CTA owns one replica for a whole kmc_run call: the replica's packed
// occupancy is staged into shared memory with TMA bulk copies
// (cp.async.bulk + mbarrier), its vacancy records are unpacked into
// shared-memory arrays linked per fragment, and the CTA runs every window and
// colour phase with __syncthreads() between phases -- no grid-wide
// synchronisation, because replicas are independent.  The fragment BKL is
// that of arXiv:2004.09081 Sec. II.A (Eqs. RateCnst1, eventSelection,
// TimeStep) with fragment-local selection (Sec. II.B, Eq. AtomP); selection
// uses exact u64 fixed-point sums, so results are identical to the
// colour-phase kernel and to the oracle's mixed form.
//
// Each colour phase has two passes:
//   screen  one thread per fragment of the colour.  A fragment whose
//           neighbourhood did not change since its last visit keeps its exact
//           event total S; with the first draw of the phase, E/S > window
//           proves that nothing happens, and the fragment is skipped.
//           Everything else goes to a compact list.
//   run     one warp per listed fragment (lane = 4 slots x 8 directions per
//           32-event chunk; the warp draws 64 events' random numbers at once):
//           exact total, clock, selection by warp scan, exchange, hand-off,
//           and "dirty" marks on the owners of every vacancy next to one of the
//           two changed sites -- exactly the fragments whose total changed.
// At the end the occupancy goes back with a TMA bulk store and the records go
// back to the per-fragment lists.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>

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

// ---- thread-block cluster and distributed shared memory
__device__ __forceinline__ uint32_t cluster_ctarank()
{
    uint32_t r;
    asm volatile("mov.u32 %0, %%cluster_ctarank;" : "=r"(r));
    return r;
}

// every thread of every CTA of the cluster; release / acquire of shared memory
__device__ __forceinline__ void cluster_sync()
{
    asm volatile("barrier.cluster.arrive.release.aligned;\n\tbarrier.cluster.wait.acquire.aligned;" ::: "memory");
}

// the two halves of cluster_sync: work that reads and writes nothing a peer
// touches may run between them
__device__ __forceinline__ void cluster_arrive()
{
    asm volatile("barrier.cluster.arrive.release.aligned;" ::: "memory");
}
__device__ __forceinline__ void cluster_wait()
{
    asm volatile("barrier.cluster.wait.acquire.aligned;" ::: "memory");
}

// address in CTA `peer`'s shared memory of the same variable as `p`
__device__ __forceinline__ uint32_t peer_addr(const void* p, uint32_t peer)
{
    uint32_t r;
    asm volatile("mapa.shared::cluster.u32 %0, %1, %2;" : "=r"(r) : "r"(smem_u32(p)), "r"(peer));
    return r;
}

__device__ __forceinline__ void st_peer(uint32_t a, uint32_t v)
{
    asm volatile("st.shared::cluster.u32 [%0], %1;" ::"r"(a), "r"(v) : "memory");
}
__device__ __forceinline__ void st_peer(uint32_t a, int32_t v) { st_peer(a, (uint32_t)v); }
__device__ __forceinline__ void st_peer16(uint32_t a, int16_t v)
{
    asm volatile("st.shared::cluster.u16 [%0], %1;" ::"r"(a), "h"((unsigned short)v) : "memory");
}
__device__ __forceinline__ void st_peer8(uint32_t a, uint8_t v)
{
    asm volatile("st.shared::cluster.u8 [%0], %1;" ::"r"(a), "h"((unsigned short)v) : "memory");
}
__device__ __forceinline__ void st_peer64(uint32_t a, unsigned long long v)
{
    asm volatile("st.shared::cluster.u64 [%0], %1;" ::"r"(a), "l"(v) : "memory");
}
__device__ __forceinline__ void red_peer_xor(uint32_t a, uint32_t v)
{
    asm volatile("red.shared::cluster.xor.b32 [%0], %1;" ::"r"(a), "r"(v) : "memory");
}
__device__ __forceinline__ int32_t atom_peer_exch(uint32_t a, int32_t v)
{
    int32_t o;
    asm volatile("atom.shared::cluster.exch.b32 %0, [%1], %2;" : "=r"(o) : "r"(a), "r"(v) : "memory");
    return o;
}
__device__ __forceinline__ uint4 ld_peer16(uint32_t a)
{
    uint4 v;
    asm volatile("ld.shared::cluster.v4.u32 {%0, %1, %2, %3}, [%4];"
                 : "=r"(v.x), "=r"(v.y), "=r"(v.z), "=r"(v.w)
                 : "r"(a)
                 : "memory");
    return v;
}
__device__ __forceinline__ int32_t ld_peer(uint32_t a)
{
    int32_t v;
    asm volatile("ld.shared::cluster.u32 %0, [%1];" : "=r"(v) : "r"(a) : "memory");
    return v;
}

constexpr uint32_t BULK_CHUNK = 32768;        // bytes per bulk copy instruction
constexpr uint64_t WAIT_NS = 2000000000ull;   // 2 s bound on any device-side wait

// compact site key in shared memory: t<<30 | z<<20 | y<<10 | x (cells < 1024),
// ordered like the linear site index
__device__ __forceinline__ uint32_t key32(int t, int x, int y, int z)
{
    return ((uint32_t)t << 30) | ((uint32_t)z << 20) | ((uint32_t)y << 10) | (uint32_t)x;
}

__device__ __forceinline__ void split32(uint32_t k, int& t, int& x, int& y, int& z)
{
    x = (int)(k & 1023u);
    y = (int)((k >> 10) & 1023u);
    z = (int)((k >> 20) & 1023u);
    t = (int)(k >> 30);
}

struct Shared {
    RepDesc D;
    NbEntry nb[3][8];
    uint64_t bar;
    uint64_t bar_test;   // the wait test's barrier, which nothing completes
    uint32_t perms[64];  // colour orders of 64 consecutive windows (nibble p = colour of phase p)
    int nv_count;
    int nact;
    int next_act;
    unsigned long long hops, hand;
    int abort;
    int cached;  // the fragment totals of the last call are valid
};

struct Layout {
    uint32_t* occ;
    uint32_t* key;
    int32_t* d;
    uint32_t* id;
    int16_t* next;
    int32_t* head;
    unsigned long long* S;
    uint8_t* dirty;
    int32_t* act;          // screened fragments
    float* pre_E;          // first exponential variates (events 0, 1, and 2, 3 where drawn) of every
    uint64_t* pre_xs;      // fragment of the batch's phases, and their selection words, by (phase in
                           // batch, screen index)
    uint16_t* frag_of_c;   // cell -> fragment index: x cells, then y, then z
    int16_t* wslot;   // per warp: vacancy index of each slot (-1: handed off)
    int8_t* wtype;    // per warp: rate type of each event (-1: none)
};


__host__ __device__ inline size_t layout_bytes(int64_t words, int64_t nv, int64_t nfrag, int64_t ncls, int cap,
                                               int nwarps, int ltot, int pre_g, int pre_ev,
                                               size_t* off /* 14 offsets or null */)
{
    // every array starts on a 16-byte boundary, whatever the sizes before it
    const size_t sz[14] = {
        (size_t)words * 4,         // 0 occupancy (bulk-copied)
        (size_t)nv * 4,            // 1 keys
        (size_t)nv * 12,           // 2 displacements
        (size_t)nv * 4,            // 3 ids
        (size_t)nv * 2,            // 4 next links
        (size_t)nfrag * 4,         // 5 list heads
        (size_t)nfrag * 8,         // 6 cached totals
        (size_t)nfrag,             // 7 dirty flags
        (size_t)ncls * 4,          // 8 screened list
        (size_t)nwarps * cap * 2,  // 9 per-warp slots
        (size_t)nwarps * cap * 8,  // 10 per-warp event types
        (size_t)pre_g * pre_ev * ncls * 8,  // 11 first draws of the batch's phases: selection words
        (size_t)pre_g * pre_ev * ncls * 4,  // 12 and variates
        (size_t)ltot * 2,          // 13 cell -> fragment tables
    };
    size_t b = 0;
    for (int k = 0; k < 14; ++k) {
        if (off) off[k] = b;
        b += (sz[k] + 15) & ~(size_t)15;
    }
    return (b + 127) & ~(size_t)127;
}

__device__ __forceinline__ Layout carve(unsigned char* dyn, int64_t words, int64_t nv, int64_t nfrag, int64_t ncls,
                                        int cap, int nwarps, int ltot, int pre_g, int pre_ev)
{
    size_t o[14];
    layout_bytes(words, nv, nfrag, ncls, cap, nwarps, ltot, pre_g, pre_ev, o);
    Layout L;
    L.occ = reinterpret_cast<uint32_t*>(dyn + o[0]);
    L.key = reinterpret_cast<uint32_t*>(dyn + o[1]);
    L.d = reinterpret_cast<int32_t*>(dyn + o[2]);
    L.id = reinterpret_cast<uint32_t*>(dyn + o[3]);
    L.next = reinterpret_cast<int16_t*>(dyn + o[4]);
    L.head = reinterpret_cast<int32_t*>(dyn + o[5]);
    L.S = reinterpret_cast<unsigned long long*>(dyn + o[6]);
    L.dirty = reinterpret_cast<uint8_t*>(dyn + o[7]);
    L.act = reinterpret_cast<int32_t*>(dyn + o[8]);
    L.pre_xs = reinterpret_cast<uint64_t*>(dyn + o[11]);
    L.pre_E = reinterpret_cast<float*>(dyn + o[12]);
    L.frag_of_c = reinterpret_cast<uint16_t*>(dyn + o[13]);
    L.wslot = reinterpret_cast<int16_t*>(dyn + o[9]);
    L.wtype = reinterpret_cast<int8_t*>(dyn + o[10]);
    return L;
}

// word and shift in the replica's occupancy of neighbour q of the site (t,x,y,z)
struct NbSite {
    int t2, jx, jy, jz;
};

// lattice sizes, row words, fragment counts, clock scale and window: loaded
// into registers once (shared-memory reads would be repeated after every
// atomic and warp barrier)
struct Geo {
    int L0, L1, L2, RW, nf0, nf1, F;
    double theta;
    float theta_f;  // the largest float <= theta 2^-F (see window_f)
};

// The window test of a clock still at zero: 2^F r > theta for the FP32 ratio r
// (2^F r is an exact double, and 0 + 2^F r is that double) holds exactly when
// r > theta 2^-F, and for a float r that holds exactly when r exceeds the
// largest float not above theta 2^-F -- one FP32 compare instead of a
// conversion, an add and a compare on the FP64 pipe, with the same outcome.
__device__ __forceinline__ float window_f(double theta, int F)
{
    return __double2float_rd(__longlong_as_double(__double_as_longlong(theta) - ((long long)F << 52)));
}

__device__ __forceinline__ NbSite nb_site(const Shared& sh, const Geo& g, int t, int x, int y, int z, int q)
{
    const NbEntry nb = sh.nb[t][q];
    NbSite s;
    s.t2 = nb.t2;
    s.jx = wrapc(x + nb.dc[0], g.L0);
    s.jy = wrapc(y + nb.dc[1], g.L1);
    s.jz = wrapc(z + nb.dc[2], g.L2);
    return s;
}

__device__ __forceinline__ int site_code(const Geo& g, const uint32_t* occ, int t, int x, int y, int z)
{
    const uint32_t w = occ[((z * g.L1 + y) * g.RW + (x >> 4)) * 3 + t];
    return (int)((w >> occ_shift(x)) & 3u);
}

// owner fragment of cell (x,y,z), from the per-dimension tables
__device__ __forceinline__ int owner_of(const Geo& g, const uint16_t* fo, int x, int y, int z)
{
    return (fo[g.L0 + g.L1 + z] * g.nf1 + fo[g.L0 + y]) * g.nf0 + fo[x];
}

// exact product 2^F * d for a positive normal double (exponent add)
__device__ __forceinline__ double scale_pow2(double d, int F)
{
    return __longlong_as_double(__double_as_longlong(d) + ((long long)F << 52));
}

}  // namespace

size_t resident_smem_bytes(const RepDesc& D, int64_t n_vac, int cap, int threads, int pre_g, int pre_ev)
{
    const int64_t words = 3 * (int64_t)D.L[2] * D.L[1] * D.row_words;
    const int64_t nfrag = (int64_t)D.nf[0] * D.nf[1] * D.nf[2];
    const int64_t ncls = (int64_t)((D.nf[0] + 1) / 2) * ((D.nf[1] + 1) / 2) * ((D.nf[2] + 1) / 2);
    if (D.L[0] > 1024 || D.L[1] > 1024 || D.L[2] > 1024 || n_vac > 32767 || nfrag > 32767)
        return ~(size_t)0;  // compact keys and 16-bit links need these bounds
    if (pre_g < 1 || pre_g > 8 || (8 % pre_g) != 0 || (pre_ev != 2 && pre_ev != 4)) return ~(size_t)0;
    return layout_bytes(words, n_vac, nfrag, ncls, cap, threads / 32, D.L[0] + D.L[1] + D.L[2], pre_g, pre_ev,
                        nullptr);
}

// CL = CTAs per replica (a thread-block cluster).  With CL = 2 both CTAs hold
// the whole replica; each screens and runs half of every colour's fragments,
// and every write to the replica's state is made in both copies (the local one
// and, through distributed shared memory, the peer's), so the copies stay
// identical; reads are local.  Phases end with a cluster barrier.
template <int NT, int CL>
__global__ void __launch_bounds__(NT, (NT <= 128 ? 4 : (NT <= 256 ? 2 : 1))) k_resident(const RepDesc* __restrict__ descs,
                                                  const int32_t* __restrict__ reps,
                                                  const int64_t* __restrict__ nvac, uint64_t windows,
                                                  uint32_t* occ, VacRec* recs, int32_t* counts,
                                                  int32_t* tracer, unsigned long long* stats,
                                                  uint32_t* status, int cap, NbTable nbt,
                                                  uint32_t stuck_wait_us, ResCache rc)
{
    extern __shared__ __align__(128) unsigned char dyn[];
    __shared__ Shared sh;
    const int tid = threadIdx.x;
    const int r = reps[blockIdx.x / CL];
    const int64_t n_vac = nvac[r];
    const uint32_t rank = CL > 1 ? cluster_ctarank() : 0u;
    const uint32_t peer = rank ^ 1u;

    if (tid == 0) {
        sh.D = descs[r];
        sh.nv_count = 0;
        sh.hops = 0;
        sh.hand = 0;
        sh.abort = 0;
        sh.cached = rc.valid[r];
    }
    if (tid < 24) (&sh.nb[0][0])[tid] = (&nbt.e[0][0])[tid];  // threads index it with different t
    __syncthreads();
    const RepDesc& D = sh.D;
    const int64_t words = 3 * (int64_t)D.L[2] * D.L[1] * D.row_words;
    const int nfrag = D.nf[0] * D.nf[1] * D.nf[2];
    const int ncls_max = ((D.nf[0] + 1) / 2) * ((D.nf[1] + 1) / 2) * ((D.nf[2] + 1) / 2);
    const int pre_g = (D.pre_g == 2 || D.pre_g == 4 || D.pre_g == 8) ? D.pre_g : 1;  // the host sized the layout for it
    const int pre_ev = D.pre_ev == 4 ? 4 : 2;  // events per fragment drawn ahead: block 0, or blocks 0 and 1
    const Layout S =
        carve(dyn, words, n_vac, nfrag, ncls_max, cap, NT / 32, D.L[0] + D.L[1] + D.L[2], pre_g, pre_ev);

    // ---- stage in: occupancy by TMA bulk copies, records by plain loads (the
    // first CTA of a cluster; the second copies its shared memory afterwards)
    const uint32_t occ_bytes = (uint32_t)(words * 4);
    if (tid == 0 && rank == 0) {
        mbar_init(&sh.bar, 1);
        mbar_arrive_expect_tx(&sh.bar, occ_bytes);
        const char* src = reinterpret_cast<const char*>(occ + D.occ_word_off);
        for (uint32_t off = 0; off < occ_bytes; off += BULK_CHUNK) {
            const uint32_t n = min(BULK_CHUNK, occ_bytes - off);
            bulk_g2s(S.occ + off / 4, src + off, n, &sh.bar);
        }
    }
    for (int k = tid; k < D.L[0] + D.L[1] + D.L[2]; k += blockDim.x) {
        const int d = k < D.L[0] ? 0 : (k < D.L[0] + D.L[1] ? 1 : 2);
        const int c = d == 0 ? k : (d == 1 ? k - D.L[0] : k - D.L[0] - D.L[1]);
        S.frag_of_c[k] = (uint16_t)frag_of(c, D.base[d], D.rem[d]);
    }
    for (int f = tid; f < (rank == 0 ? nfrag : 0); f += blockDim.x) {
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
            int t, x, y, z;
            split_key(rr.key, t, x, y, z);
            S.key[v] = key32(t, x, y, z);
            S.d[3 * v] = rr.d[0];
            S.d[3 * v + 1] = rr.d[1];
            S.d[3 * v + 2] = rr.d[2];
            S.id[v] = rr.id;
            S.next[v] = (int16_t)head;
            head = v;
        }
        if (c > cap) atomicOr(status, STATUS_OVERFLOW);
        S.head[f] = head;
        // the fragment totals the last call left, where nothing changed the replica since
        S.dirty[f] = sh.cached ? rc.dirty[g] : 1;
        S.S[f] = sh.cached ? rc.tot[g] : 0ull;
    }
    __syncthreads();  // the barrier init is visible to every thread from here on
    if (rank == 0 && !mbar_wait_bounded(&sh.bar, 0, WAIT_NS)) {
        if (tid == 0) {
            atomicOr(status, STATUS_TIMEOUT);
            sh.abort = 1;
        }
        mbar_wait_bounded(&sh.bar, 0, WAIT_NS);  // let copies in flight land before leaving
    }
    __syncthreads();
    if (stuck_wait_us && rank == 0 && !sh.abort) {
        // test of the bounded wait: no copy is in flight here, and the barrier
        // below is never completed, so the wait must give up after
        // stuck_wait_us, report FKMC_ETIMEOUT and leave the state untouched
        if (tid == 0) mbar_init(&sh.bar_test, 1);
        __syncthreads();
        const bool done = mbar_wait_bounded(&sh.bar_test, 0, (uint64_t)stuck_wait_us * 1000ull);
        if (!done && tid == 0) {
            atomicOr(status, STATUS_TIMEOUT);
            sh.abort = 1;
        }
        __syncthreads();
    }
    if constexpr (CL > 1) {
        // every CTA of the cluster passes the same barriers: the decision to stop
        // is read from the first CTA after the cluster barrier
        cluster_sync();
        if (rank != 0) {
            if (tid == 0) sh.abort = ld_peer(peer_addr(&sh.abort, 0));
            __syncthreads();
            if (!sh.abort) {
                const uint32_t base = peer_addr(dyn, 0);
                const size_t bytes = layout_bytes(words, n_vac, nfrag, ncls_max, cap, NT / 32,
                                                  D.L[0] + D.L[1] + D.L[2], pre_g, pre_ev, nullptr);
                for (size_t k = (size_t)tid * 16; k < bytes; k += (size_t)NT * 16) {
                    const uint4 v = ld_peer16(base + (uint32_t)k);
                    *reinterpret_cast<uint4*>(dyn + k) = v;
                }
            }
        }
        cluster_sync();  // the first CTA writes into the copy only after it is complete
    }
    if (sh.abort) return;

    const uint64_t hop_k1 = key_word(D.replica, PURPOSE_HOP);
    const Geo geo{D.L[0], D.L[1], D.L[2], D.row_words, D.nf[0], D.nf[1], D.F, D.theta_tau, window_f(D.theta_tau, D.F)};
    const int lane = tid & 31;
    const int warp = tid >> 5;
    const unsigned FULL = 0xffffffffu;
    int16_t* wslot = S.wslot + warp * cap;
    int8_t* wtype = S.wtype + warp * cap * 8;
    unsigned long long my_hops = 0, my_hand = 0;

    for (uint64_t wk = 0; wk < windows; ++wk) {
        const uint64_t w = D.window + wk;
        if ((wk & 63) == 0) {  // colour orders of the next 64 windows, one thread each
            if (tid < 64 && wk + tid < windows) sh.perms[tid] = colour_perm_packed(D.seed, D.replica, w + tid);
            __syncthreads();
        }
        const uint32_t wperm = sh.perms[wk & 63];
        for (int p = 0; p < 8; ++p) {
            const int colour = (int)((wperm >> (4 * p)) & 15u);
            int cnt[3], bit[3];
#pragma unroll
            for (int d = 0; d < 3; ++d) {
                bit[d] = (colour >> d) & 1;
                cnt[d] = D.nf[d] == 1 ? (bit[d] == 0 ? 1 : 0) : D.nf[d] / 2;
            }
            const int ncls = cnt[0] * cnt[1] * cnt[2];
            const int pslot = p & (pre_g - 1);  // this phase's rows of the first-draw arrays
            if (pslot == 0) {
                // first draws (block 0: events 0 and 1; with pre_ev 4 also block 1: events 2
                // and 3) of every fragment of the next pre_g phases, one thread per block:
                // they depend on no state, and one batch of Philox blocks here replaces one
                // per phase (and one per visit of two events or more) on the critical paths
                const int nbk = pre_ev >> 1;
                for (int it = tid; it < pre_g * ncls_max * nbk; it += NT) {
                    const int idx = nbk == 2 ? it >> 1 : it, bk = it - idx * nbk;
                    const int pp = idx / ncls_max, l = idx - pp * ncls_max;
                    const int col = (int)((wperm >> (4 * (p + pp))) & 15u);
                    int c3[3], f3[3];
#pragma unroll
                    for (int d = 0; d < 3; ++d)
                        c3[d] = D.nf[d] == 1 ? (((col >> d) & 1) == 0 ? 1 : 0) : D.nf[d] / 2;
                    if (l >= c3[0] * c3[1] * c3[2]) continue;
                    f3[0] = l % c3[0];
                    f3[1] = (l / c3[0]) % c3[1];
                    f3[2] = l / (c3[0] * c3[1]);
#pragma unroll
                    for (int d = 0; d < 3; ++d) f3[d] = D.nf[d] == 1 ? 0 : 2 * f3[d] + ((col >> d) & 1);
                    const int fid = (f3[2] * D.nf[1] + f3[1]) * D.nf[0] + f3[0];
                    const U64x4 blk = philox4x64((uint64_t)fid, w, (uint64_t)bk, 0, D.seed, hop_k1);
                    const int o = pre_ev * idx + 2 * bk;
                    S.pre_E[o] = neglog32(blk.x[0]);
                    S.pre_E[o + 1] = neglog32(blk.x[2]);
                    S.pre_xs[o] = blk.x[1];
                    S.pre_xs[o + 1] = blk.x[3];
                }
            }
            if (tid == 0) {
                sh.nact = 0;
                sh.next_act = 0;
            }
            __syncthreads();
            // ---- screen: one thread per fragment of the colour
            for (int l = tid * CL + (int)rank; l < ncls; l += NT * CL) {
                int f0 = l % cnt[0], f1 = (l / cnt[0]) % cnt[1], f2 = l / (cnt[0] * cnt[1]);
                f0 = D.nf[0] == 1 ? 0 : 2 * f0 + bit[0];
                f1 = D.nf[1] == 1 ? 0 : 2 * f1 + bit[1];
                f2 = D.nf[2] == 1 ? 0 : 2 * f2 + bit[2];
                const int fid = (f2 * D.nf[1] + f1) * D.nf[0] + f0;
                if (S.head[fid] < 0) continue;
                const bool dirty = S.dirty[fid] != 0;
                const unsigned long long tot = S.S[fid];
                if (!dirty && tot == 0ull) continue;
                bool active = dirty;
                if (!active) {
                    const float E0 = S.pre_E[pre_ev * (pslot * ncls_max + l)];
                    const float ratio = __fdiv_rn(E0, __ull2float_rn(tot));
                    active = !(ratio > geo.theta_f);  // 0 + 2^F ratio <= theta
                }
                if (active) {
                    const int a = atomicAdd(&sh.nact, 1);
                    S.act[a] = f0 | (f1 << 10) | (f2 << 20);  // fragment coordinates (< 1024 each)
                }
            }
            __syncthreads();
            // ---- run: one warp per listed fragment
            const int nact = sh.nact;
            for (;;) {
                // warps take the screened fragments one at a time, as they become free
                int a = 0;
                if (lane == 0) a = atomicAdd(&sh.next_act, 1);
                a = __shfl_sync(FULL, a, 0);
                if (a >= nact) break;
                const int fxyz = S.act[a];
                const int fx = fxyz & 1023, fy = (fxyz >> 10) & 1023, fz = fxyz >> 20;
                const int fid = (fz * D.nf[1] + fy) * D.nf[0] + fx;
                // the fragment's screen index within its colour, and its row of first draws
                const int ls = ((D.nf[2] == 1 ? 0 : fz >> 1) * cnt[1] + (D.nf[1] == 1 ? 0 : fy >> 1)) * cnt[0] +
                               (D.nf[0] == 1 ? 0 : fx >> 1);
                const int prow = pslot * ncls_max + ls;
                const int lo0 = frag_start(fx, D.base[0], D.rem[0]), hi0 = frag_start(fx + 1, D.base[0], D.rem[0]);
                const int lo1 = frag_start(fy, D.base[1], D.rem[1]), hi1 = frag_start(fy + 1, D.base[1], D.rem[1]);
                const int lo2 = frag_start(fz, D.base[2], D.rem[2]), hi2 = frag_start(fz + 1, D.base[2], D.rem[2]);
                // slots: the fragment's vacancies in ascending site order
                int n = 0;
                if (lane == 0) {
                    for (int v = S.head[fid]; v >= 0; v = S.next[v]) {
                        if (n >= cap) {
                            atomicOr(status, STATUS_OVERFLOW);
                            break;
                        }
                        wslot[n++] = (int16_t)v;
                    }
                }
                n = __shfl_sync(FULL, n, 0);
                __syncwarp();
                // a list that received no vacancy since its last visit is still in site order
                bool ordered = false;
                uint32_t kk = 0xffffffffu;
                if (n <= 32) {  // rank by site (sites are distinct), unless already in order
                    const int vk = lane < n ? wslot[lane] : -1;
                    kk = lane < n ? S.key[vk] : 0xffffffffu;
                    const uint32_t kprev = __shfl_up_sync(FULL, kk, 1);
                    ordered = __ballot_sync(FULL, lane > 0 && lane < n && kprev > kk) == 0u;
                    if (!ordered) {
                        int rnk = 0;
                        for (int q = 0; q < n; ++q) rnk += __shfl_sync(FULL, kk, q) < kk ? 1 : 0;
                        __syncwarp();
                        if (lane < n) wslot[rnk] = (int16_t)vk;
                    }
                } else if (lane == 0) {
                    for (int k = 1; k < n; ++k) {
                        const int v = wslot[k];
                        const uint32_t kv = S.key[v];
                        int m = k;
                        while (m > 0 && S.key[wslot[m - 1]] > kv) {
                            wslot[m] = wslot[m - 1];
                            --m;
                        }
                        wslot[m] = (int16_t)v;
                    }
                }
                __syncwarp();
                const int nch = (n + 3) >> 2;
                // up to two chunks (8 vacancies): each lane keeps the site keys of its two
                // events' slots in registers (0xffffffff: no slot, or handed off)
                uint32_t kc0 = 0xffffffffu, kc1 = 0xffffffffu;
                if (nch <= 2) {
                    const int m0 = lane >> 3, m1 = 4 + (lane >> 3);
                    if (ordered) {  // lane m holds slot m's key
                        const uint32_t a0 = __shfl_sync(FULL, kk, m0), a1 = __shfl_sync(FULL, kk, m1);
                        if (m0 < n) kc0 = a0;
                        if (m1 < n) kc1 = a1;
                    } else {
                        if (m0 < n) kc0 = S.key[wslot[m0]];
                        if (m1 < n) kc1 = S.key[wslot[m1]];
                    }
                }
                auto type_of = [&](uint32_t k, int q) -> int {
                    int t, x, y, z;
                    split32(k, t, x, y, z);
                    const NbEntry nbe = sh.nb[t][q];
                    const int code = site_code(geo, S.occ, nbe.t2, wrapc(x + nbe.dc[0], geo.L0),
                                               wrapc(y + nbe.dc[1], geo.L1), wrapc(z + nbe.dc[2], geo.L2));
                    return code == SP_V ? -1 : code * 3 + nbe.d[2] + 1;
                };
                int ty0 = -1, ty1 = -1;  // up to two chunks: rate types of events lane and 32 + lane
                auto compute_types = [&]() {
                    if (nch <= 2) {
                        ty0 = kc0 != 0xffffffffu ? type_of(kc0, lane & 7) : -1;
                        ty1 = (nch == 2 && kc1 != 0xffffffffu) ? type_of(kc1, lane & 7) : -1;
                    } else {
                        for (int c = 0; c < nch; ++c) {
                            const int e = c * 32 + lane, m = e >> 3;
                            int ty = -1;
                            if (m < n && wslot[m] >= 0) ty = type_of(S.key[wslot[m]], e & 7);
                            wtype[e] = (int8_t)ty;
                        }
                    }
                    __syncwarp();
                };
                compute_types();

                double clock = 0.0;
                uint64_t i = 0, batch = ~0ull;
                uint64_t xs_even = 0, xs_odd = 0;
                float E_even = 0.f, E_odd = 0.f;
                unsigned long long tot = 0;
                for (;;) {
                    // exact total of the fragment's events (order-free integer sum).  Up to two
                    // chunks (8 vacancies) one inclusive scan gives both the total and the
                    // prefixes the selection needs; beyond that, a reduction now and scans later.
                    unsigned long long inc0 = 0, inc1 = 0;
                    if (nch <= 2) {
                        const int t0 = ty0;
                        inc0 = t0 < 0 ? 0ull : (unsigned long long)D.q[t0];
#pragma unroll
                        for (int off = 1; off < 32; off <<= 1) {
                            const unsigned long long t2 = __shfl_up_sync(FULL, inc0, off);
                            if (lane >= off) inc0 += t2;
                        }
                        tot = __shfl_sync(FULL, inc0, 31);
                        if (nch == 2) {
                            const int t1 = ty1;
                            inc1 = t1 < 0 ? 0ull : (unsigned long long)D.q[t1];
#pragma unroll
                            for (int off = 1; off < 32; off <<= 1) {
                                const unsigned long long t2 = __shfl_up_sync(FULL, inc1, off);
                                if (lane >= off) inc1 += t2;
                            }
                            inc1 += tot;
                            tot = __shfl_sync(FULL, inc1, 31);
                        }
                    } else {
                        unsigned long long part = 0;
                        for (int c = 0; c < nch; ++c) {
                            const int ty = wtype[c * 32 + lane];
                            part += ty < 0 ? 0ull : (unsigned long long)D.q[ty];
                        }
#pragma unroll
                        for (int off = 16; off; off >>= 1) part += __shfl_xor_sync(FULL, part, off);
                        tot = part;
                    }
                    if (tot == 0ull) break;
                    if (i >= MAX_EVENTS_PER_PHASE) {
                        if (lane == 0) atomicOr(status, STATUS_EVENT_LIMIT);
                        break;
                    }
                    uint64_t xs;
                    float E;
                    if (i < (uint64_t)pre_ev) {  // blocks 0 (and 1), drawn in the batch before the phase
                        xs = S.pre_xs[pre_ev * prow + (int)i];
                        E = S.pre_E[pre_ev * prow + (int)i];
                    } else {
                        // events [2 + 64 b, 66 + 64 b) come from blocks 1 + 32 b + lane (block 1,
                        // events 2 and 3, was drawn ahead with pre_ev 4: lane 0 recomputes it unused)
                        const uint64_t k = i - 2;
                        if ((k >> 6) != batch) {
                            batch = k >> 6;
                            const U64x4 blk =
                                philox4x64((uint64_t)fid, w, 1 + 32 * batch + lane, 0, D.seed, hop_k1);
                            xs_even = blk.x[1];
                            xs_odd = blk.x[3];
                            E_even = neglog32(blk.x[0]);
                            E_odd = neglog32(blk.x[2]);
                        }
                        const int src = (int)((k >> 1) & 31);
                        const bool odd = (k & 1) != 0;
                        xs = __shfl_sync(FULL, odd ? xs_odd : xs_even, src);
                        E = __shfl_sync(FULL, odd ? E_odd : E_even, src);
                    }
                    const float ratio = __fdiv_rn(E, __ull2float_rn(tot));
                    const double nclock = __dadd_rn(clock, scale_pow2((double)ratio, geo.F));
                    const bool past = i == 0 ? ratio > geo.theta_f : nclock > geo.theta;  // the first: clock 0
                    // up to two chunks: the selection (no side effects) before the clock test,
                    // so that its shuffles overlap the clock's FP64 chain; a break discards it
                    const unsigned long long target = __umul64hi(xs, tot);
                    int e_sel = -1;
                    uint32_t ksel = 0u;
                    int tsel = -1;
                    if (nch <= 2) {
                        unsigned bal = __ballot_sync(FULL, inc0 > target);
                        if (bal) {
                            e_sel = __ffs(bal) - 1;
                        } else {
                            bal = __ballot_sync(FULL, inc1 > target);
                            if (bal && nch == 2) e_sel = 32 + __ffs(bal) - 1;
                        }
                        const int ms = e_sel >> 3;  // the slot's site key and the event's type
                        ksel = __shfl_sync(FULL, ms < 4 ? kc0 : kc1, (ms & 3) << 3);
                        tsel = __shfl_sync(FULL, e_sel < 32 ? ty0 : ty1, e_sel & 31);
                    }
                    if (past) break;
                    // first event whose running sum exceeds the target
                    if (nch > 2) {
                        unsigned long long carry = 0;
                        for (int c = 0; c < nch; ++c) {
                            const int ty = wtype[c * 32 + lane];
                            unsigned long long inc = ty < 0 ? 0ull : (unsigned long long)D.q[ty];
#pragma unroll
                            for (int off = 1; off < 32; off <<= 1) {
                                const unsigned long long t2 = __shfl_up_sync(FULL, inc, off);
                                if (lane >= off) inc += t2;
                            }
                            inc += carry;
                            const unsigned bal = __ballot_sync(FULL, inc > target);
                            if (bal) {
                                e_sel = c * 32 + __ffs(bal) - 1;
                                break;
                            }
                            carry = __shfl_sync(FULL, inc, 31);
                        }
                    }
                    if (e_sel < 0) {  // cannot happen: the target lies below the total
                        if (lane == 0) atomicOr(status, STATUS_OVERFLOW);
                        break;
                    }
                    const int m = e_sel >> 3, qd = e_sel & 7;
                    int t, x, y, z;
                    split32(nch <= 2 ? ksel : S.key[wslot[m]], t, x, y, z);
                    const NbEntry nb = sh.nb[t][qd];
                    const NbSite j = nb_site(sh, geo, t, x, y, z, qd);
                    const bool owned = j.jx >= lo0 && j.jx < hi0 && j.jy >= lo1 && j.jy < hi1 && j.jz >= lo2 &&
                                       j.jz < hi2;
                    if (lane == 0) {  // apply the exchange
                        const int v = wslot[m];
                        const uint32_t ion = (uint32_t)((nch <= 2 ? tsel : (int)wtype[e_sel]) / 3);
                        uint32_t* ws = S.occ + ((z * geo.L1 + y) * geo.RW + (x >> 4)) * 3 + t;
                        uint32_t* wj = S.occ + ((j.jz * geo.L1 + j.jy) * geo.RW + (j.jx >> 4)) * 3 + j.t2;
                        const uint32_t ms = ((uint32_t)SP_V ^ ion) << occ_shift(x);
                        const uint32_t mj = (ion ^ (uint32_t)SP_V) << occ_shift(j.jx);
                        atomicXor(ws, ms);
                        atomicXor(wj, mj);
                        S.d[3 * v] += nb.d[0];
                        S.d[3 * v + 1] += nb.d[1];
                        S.d[3 * v + 2] += nb.d[2];
                        if constexpr (CL > 1) {
                            red_peer_xor(peer_addr(ws, peer), ms);
                            red_peer_xor(peer_addr(wj, peer), mj);
                            for (int k = 0; k < 3; ++k) st_peer(peer_addr(S.d + 3 * v + k, peer), S.d[3 * v + k]);
                        }
                        if (tracer) {
                            const int64_t s_lin = (((int64_t)t * D.L[2] + z) * D.L[1] + y) * D.L[0] + x;
                            const int64_t j_lin = (((int64_t)j.t2 * D.L[2] + j.jz) * D.L[1] + j.jy) * D.L[0] + j.jx;
                            int32_t* ts = tracer + 3 * (D.site_off + s_lin);
                            int32_t* tj = tracer + 3 * (D.site_off + j_lin);
                            ts[0] = tj[0] - nb.d[0];
                            ts[1] = tj[1] - nb.d[1];
                            ts[2] = tj[2] - nb.d[2];
                            tj[0] = tj[1] = tj[2] = 0;
                        }
                        S.key[v] = key32(j.t2, j.jx, j.jy, j.jz);
                        if constexpr (CL > 1) st_peer(peer_addr(S.key + v, peer), S.key[v]);
                        if (!owned) {
                            // leaves the fragment: its slot goes dead (zero rate), the record
                            // is pushed onto the owner's list (the owner does not run in this
                            // phase, so that list only receives pushes; links are read after
                            // the phase barrier)
                            wslot[m] = -1;
                            const int g2 = owner_of(geo, S.frag_of_c, j.jx, j.jy, j.jz);
                            S.next[v] = (int16_t)atomicExch(S.head + g2, v);
                            if constexpr (CL > 1)
                                st_peer16(peer_addr(S.next + v, peer),
                                          (int16_t)atom_peer_exch(peer_addr(S.head + g2, peer), v));
                            ++my_hand;
                        }
                    }
                    __syncwarp();
                    if (nch <= 2) {  // the moved vacancy's lanes follow it (or drop a handed-off slot)
                        const uint32_t nk = owned ? key32(j.t2, j.jx, j.jy, j.jz) : 0xffffffffu;
                        if ((lane >> 3) == m) kc0 = nk;
                        if (4 + (lane >> 3) == m) kc1 = nk;
                    }
                    {
                        // the fragments whose totals changed: owners of the vacancies next to the
                        // two changed sites (lanes 0-7 look around s, 8-15 around j; 16-31 repeat
                        // them without storing, so that no branch splits the warp and the probe's
                        // loads overlap those of the rate types)
                        const int pl = lane & 15;
                        const int bt = pl < 8 ? t : j.t2;
                        const int bx = pl < 8 ? x : j.jx, by = pl < 8 ? y : j.jy, bz = pl < 8 ? z : j.jz;
                        const NbSite c = nb_site(sh, geo, bt, bx, by, bz, pl & 7);
                        const bool vac = site_code(geo, S.occ, c.t2, c.jx, c.jy, c.jz) == SP_V;
                        const int g = owner_of(geo, S.frag_of_c, c.jx, c.jy, c.jz);
                        compute_types();
                        if (lane < 16 && vac && g != fid) {
                            S.dirty[g] = 1;
                            if constexpr (CL > 1) st_peer8(peer_addr(S.dirty + g, peer), 1);
                        }
                    }
                    clock = nclock;
                    ++i;
                }
                // surviving vacancies stay linked to this fragment, in slot order (up to 32
                // slots, each lane links its own slot to the next live one)
                int head = -1;
                if (n <= 32) {
                    const int v = lane < n ? wslot[lane] : -1;
                    const unsigned live = __ballot_sync(FULL, v >= 0);
                    const unsigned later = live & ~((2u << lane) - 1u);
                    const int vn = __shfl_sync(FULL, v, later ? __ffs(later) - 1 : 0);
                    const int hv = __shfl_sync(FULL, v, live ? __ffs(live) - 1 : 0);
                    if (v >= 0) {
                        S.next[v] = (int16_t)(later ? vn : -1);
                        if constexpr (CL > 1) st_peer16(peer_addr(S.next + v, peer), (int16_t)(later ? vn : -1));
                    }
                    head = live ? hv : -1;
                }
                if (lane == 0) {
                    if (n > 32) {
                        for (int m = n - 1; m >= 0; --m) {
                            const int v = wslot[m];
                            if (v < 0) continue;
                            S.next[v] = (int16_t)head;
                            if constexpr (CL > 1) st_peer16(peer_addr(S.next + v, peer), (int16_t)head);
                            head = v;
                        }
                    }
                    S.head[fid] = head;
                    S.S[fid] = tot;
                    S.dirty[fid] = 0;
                    if constexpr (CL > 1) {
                        st_peer(peer_addr(S.head + fid, peer), head);
                        st_peer64(peer_addr(S.S + fid, peer), tot);
                        st_peer8(peer_addr(S.dirty + fid, peer), 0);
                    }
                    my_hops += i;
                }
                __syncwarp();
            }
            if constexpr (CL > 1) cluster_sync();  // both copies hold every write of the phase
            else __syncthreads();
        }
    }

    // ---- stage out (the first CTA of a cluster): occupancy by a TMA bulk store, records to the fragment lists
    if (tid == 0 && rank == 0) {
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        char* dst = reinterpret_cast<char*>(occ + D.occ_word_off);
        for (uint32_t off = 0; off < occ_bytes; off += BULK_CHUNK) {
            const uint32_t nb = min(BULK_CHUNK, occ_bytes - off);
            bulk_s2g(dst + off, S.occ + off / 4, nb);
        }
        asm volatile("cp.async.bulk.commit_group;" ::: "memory");
    }
    for (int f = tid; f < (rank == 0 ? nfrag : 0); f += blockDim.x) {
        const int64_t g = D.frag_base + f;
        int k = 0;
        for (int v = S.head[f]; v >= 0; v = S.next[v], ++k) {
            if (k >= cap) {
                atomicOr(status, STATUS_OVERFLOW);
                break;
            }
            int t, x, y, z;
            split32(S.key[v], t, x, y, z);
            VacRec rr;
            rr.key = make_key(t, x, y, z);
            rr.d[0] = S.d[3 * v];
            rr.d[1] = S.d[3 * v + 1];
            rr.d[2] = S.d[3 * v + 2];
            rr.id = S.id[v];
            recs[g * cap + k] = rr;
        }
        counts[g] = k;
        rc.tot[g] = S.S[f];
        rc.dirty[g] = S.dirty[f];
    }
    atomicAdd(&sh.hops, my_hops);
    atomicAdd(&sh.hand, my_hand);
    __syncthreads();
    if (tid == 0) {
        if (sh.hops) atomicAdd(stats + 2 * r, sh.hops);
        if (sh.hand) atomicAdd(stats + 2 * r + 1, sh.hand);
        if (rank == 0) {
            asm volatile("cp.async.bulk.wait_group 0;" ::: "memory");
            rc.valid[r] = 1;
        }
    }
    if constexpr (CL > 1) cluster_sync();  // no CTA leaves while its peer may still address it
}

// ---------------------------------------------------------------- cluster-resident kernel
// One replica too large for one SM's shared memory, held by a thread-block
// cluster of P.ncta CTAs (up to 16): CTA c holds the z-slab of fragment layers
// [P.fz0[c], P.fz0[c+1]) -- its occupancy planes, its vacancies (a pool of
// P.vcap slots with a free-slot stack) and its fragments' lists, totals and
// dirty flags.  Every CTA has the same layout, so a peer's copy of an array is
// addressed through distributed shared memory (mapa) at the same offset.  The
// colour phases are those of the replica-resident kernel, with a cluster
// barrier between phases:
//   - a neighbour site in another slab is read from that CTA's shared memory
//     (ld.shared::cluster), an exchange there is an atomic XOR on it
//     (red.shared::cluster);
//   - a vacancy leaving the slab is written into the owning CTA's inbox
//     (double-buffered by phase parity; the slot taken with a remote atomic
//     add) and its slot returns to the free stack; at the start of the next
//     phase the owner moves its inbox into free slots and onto the fragments'
//     lists (the receiving fragment has another colour, so it does not run in
//     the phase that filled the inbox);
//   - dirty marks on a peer's fragments are remote byte stores.
// Fragments of one colour never touch each other's sites, so the result is
// the replica-resident kernel's (and the oracle's) bit for bit.

struct InboxRec {
    uint32_t key;
    int32_t d[3];
    uint32_t id;
    int32_t lf;  // the receiving CTA's local fragment index
};
static_assert(sizeof(InboxRec) == 24, "inbox record");

struct CShared {
    RepDesc D;
    NbEntry nb[3][8];
    ClusterPlan P;
    uint32_t perms[64];
    int zbeg[CLUSTER_MAX_CTAS + 1];  // first z cell of CTA c's slab
    int nact;
    int next_act;
    int inbox_n[2];
    int free_top;
    int pool_n;
    int cached;  // the fragment totals of the last call are valid
    unsigned long long hops, hand;
};

struct CLayout {
    uint32_t* occ;       // [zs][L1][RW][3], the global layout of the slab's z cells
    uint32_t* key;       // vacancy pool [vcap]
    int32_t* d;
    uint32_t* id;
    int16_t* next;
    int16_t* fstack;     // free pool slots
    int32_t* head;       // local fragments [nfl]
    unsigned long long* S;
    uint8_t* dirty;
    int32_t* act;        // screened local fragments, with their first draws
    uint64_t* act_xs;
    float* act_E;
    int16_t* wslot;      // per warp
    int8_t* wtype;
    InboxRec* inbox;     // [2][icap]
    uint16_t* frag_of_c; // cell -> global fragment coordinate: x cells, then y, then z
    uint32_t* zmap;      // z cell -> its CTA | z within that CTA's slab << 8 | fragment layer within it << 18
    uint64_t* pre_xs;    // the next phase's first draws by screen index: selection words of events 0, 1
    float* pre_E;        // and their exponential variates
};

__host__ __device__ inline size_t cluster_layout_bytes(const RepDesc& D, const ClusterPlan& P, int cap, int nwarps,
                                                       size_t* off /* 19 offsets or null */)
{
    const size_t words = (size_t)3 * P.zs * D.L[1] * D.row_words;
    const size_t sz[19] = {
        words * 4,                          // 0 occupancy slab
        (size_t)P.vcap * 4,                 // 1 keys
        (size_t)P.vcap * 12,                // 2 displacements
        (size_t)P.vcap * 4,                 // 3 ids
        (size_t)P.vcap * 2,                 // 4 next links
        (size_t)P.vcap * 2,                 // 5 free-slot stack
        (size_t)P.nfl * 4,                  // 6 list heads
        (size_t)P.nfl * 8,                  // 7 cached totals
        (size_t)P.nfl,                      // 8 dirty flags
        (size_t)P.nfl * 4,                  // 9 screened list
        (size_t)P.nfl * 16,                 // 10 screened: selection words
        (size_t)P.nfl * 8,                  // 11 screened: variates
        (size_t)nwarps * cap * 2,           // 12 per-warp slots
        (size_t)nwarps * cap * 8,           // 13 per-warp event types
        (size_t)2 * P.icap * sizeof(InboxRec),  // 14 inboxes
        (size_t)(D.L[0] + D.L[1] + D.L[2]) * 2, // 15 cell -> fragment tables
        (size_t)D.L[2] * 4,                 // 16 z cell -> CTA, slab z, slab fragment layer
        (size_t)P.nfl * 16,                 // 17 next phase: selection words of events 0, 1
        (size_t)P.nfl * 8,                  // 18 next phase: variates
    };
    size_t b = 0;
    for (int k = 0; k < 19; ++k) {
        if (off) off[k] = b;
        b += (sz[k] + 15) & ~(size_t)15;
    }
    return (b + 127) & ~(size_t)127;
}

namespace {

__device__ __forceinline__ CLayout ccarve(unsigned char* dyn, const RepDesc& D, const ClusterPlan& P, int cap,
                                          int nwarps)
{
    size_t o[19];
    cluster_layout_bytes(D, P, cap, nwarps, o);
    CLayout L;
    L.occ = reinterpret_cast<uint32_t*>(dyn + o[0]);
    L.key = reinterpret_cast<uint32_t*>(dyn + o[1]);
    L.d = reinterpret_cast<int32_t*>(dyn + o[2]);
    L.id = reinterpret_cast<uint32_t*>(dyn + o[3]);
    L.next = reinterpret_cast<int16_t*>(dyn + o[4]);
    L.fstack = reinterpret_cast<int16_t*>(dyn + o[5]);
    L.head = reinterpret_cast<int32_t*>(dyn + o[6]);
    L.S = reinterpret_cast<unsigned long long*>(dyn + o[7]);
    L.dirty = reinterpret_cast<uint8_t*>(dyn + o[8]);
    L.act = reinterpret_cast<int32_t*>(dyn + o[9]);
    L.act_xs = reinterpret_cast<uint64_t*>(dyn + o[10]);
    L.act_E = reinterpret_cast<float*>(dyn + o[11]);
    L.wslot = reinterpret_cast<int16_t*>(dyn + o[12]);
    L.wtype = reinterpret_cast<int8_t*>(dyn + o[13]);
    L.inbox = reinterpret_cast<InboxRec*>(dyn + o[14]);
    L.frag_of_c = reinterpret_cast<uint16_t*>(dyn + o[15]);
    L.zmap = reinterpret_cast<uint32_t*>(dyn + o[16]);
    L.pre_xs = reinterpret_cast<uint64_t*>(dyn + o[17]);
    L.pre_E = reinterpret_cast<float*>(dyn + o[18]);
    return L;
}

__device__ __forceinline__ uint32_t atom_peer_add(uint32_t a, uint32_t v)
{
    uint32_t o;
    asm volatile("atom.shared::cluster.add.u32 %0, [%1], %2;" : "=r"(o) : "r"(a), "r"(v) : "memory");
    return o;
}

__device__ __forceinline__ uint32_t cluster_nctas()
{
    uint32_t r;
    asm volatile("mov.u32 %0, %%cluster_nctarank;" : "=r"(r));
    return r;
}

// where a site's occupancy word lives: the CTA holding its z, and the word's
// index in that CTA's slab (every CTA has the same slab layout)
struct CWord {
    uint32_t cta;
    int idx;
};

__device__ __forceinline__ CWord cword(const CLayout& S, const Geo& g, int t, int x, int y, int z)
{
    const uint32_t zm = S.zmap[z];
    CWord w;
    w.cta = zm & 255u;
    w.idx = ((((int)((zm >> 8) & 1023u)) * g.L1 + y) * g.RW + (x >> 4)) * 3 + t;
    return w;
}

__device__ __forceinline__ int csite_code(const CLayout& S, const Geo& g, uint32_t me, int t, int x, int y, int z)
{
    const CWord w = cword(S, g, t, x, y, z);
    const uint32_t v = w.cta == me ? S.occ[w.idx] : (uint32_t)ld_peer(peer_addr(S.occ + w.idx, w.cta));
    return (int)((v >> occ_shift(x)) & 3u);
}

__device__ __forceinline__ void csite_xor(const CLayout& S, const Geo& g, uint32_t me, int t, int x, int y, int z,
                                          uint32_t m)
{
    const CWord w = cword(S, g, t, x, y, z);
    if (w.cta == me) atomicXor(S.occ + w.idx, m);
    else red_peer_xor(peer_addr(S.occ + w.idx, w.cta), m);
}

__device__ __forceinline__ NbSite cnb_site(const CShared& sh, const Geo& g, int t, int x, int y, int z, int q)
{
    const NbEntry nb = sh.nb[t][q];
    NbSite s;
    s.t2 = nb.t2;
    s.jx = wrapc(x + nb.dc[0], g.L0);
    s.jy = wrapc(y + nb.dc[1], g.L1);
    s.jz = wrapc(z + nb.dc[2], g.L2);
    return s;
}

// owner of cell (x,y,z): its CTA and that CTA's local fragment index
__device__ __forceinline__ void cowner(const CLayout& S, const Geo& g, int x, int y, int z, uint32_t& cta, int& lf)
{
    const int fx = S.frag_of_c[x], fy = S.frag_of_c[g.L0 + y];
    const uint32_t zm = S.zmap[z];
    cta = zm & 255u;
    lf = ((int)(zm >> 18) * g.nf1 + fy) * g.nf0 + fx;
}

}  // namespace

template <int NT>
__global__ void __launch_bounds__(NT, 1) k_cluster(const RepDesc* __restrict__ descs,
                                                   const ClusterPlan* __restrict__ plans, uint64_t windows,
                                                   uint32_t* occ, VacRec* recs, int32_t* counts, int32_t* tracer,
                                                   unsigned long long* stats, uint32_t* status, int cap, NbTable nbt,
                                                   ResCache rc)
{
    extern __shared__ __align__(128) unsigned char dyn[];
    __shared__ CShared sh;
    const int tid = threadIdx.x;
    const uint32_t me = cluster_ctarank();
    const int ci = (int)(blockIdx.x / cluster_nctas());
    if (tid == 0) {
        sh.P = plans[ci];
        sh.D = descs[sh.P.rep];
        for (int c = 0; c <= sh.P.ncta; ++c) sh.zbeg[c] = frag_start(sh.P.fz0[c], sh.D.base[2], sh.D.rem[2]);
        sh.nact = 0;
        sh.next_act = 0;
        sh.inbox_n[0] = sh.inbox_n[1] = 0;
        sh.pool_n = 0;
        sh.hops = 0;
        sh.hand = 0;
        sh.cached = rc.valid[sh.P.rep];
    }
    if (tid < 24) (&sh.nb[0][0])[tid] = (&nbt.e[0][0])[tid];
    __syncthreads();
    const RepDesc& D = sh.D;
    const ClusterPlan& P = sh.P;
    const CLayout S = ccarve(dyn, D, P, cap, NT / 32);
    const Geo geo{D.L[0], D.L[1], D.L[2], D.row_words, D.nf[0], D.nf[1], D.F, D.theta_tau, window_f(D.theta_tau, D.F)};
    const int fzb = P.fz0[me], fze = P.fz0[me + 1];
    const int zb = sh.zbeg[me], zl = sh.zbeg[me + 1] - zb;
    const int nfl_me = (fze - fzb) * D.nf[0] * D.nf[1];

    // ---- stage in: this slab's occupancy (its z cells are contiguous in the
    // global layout), its vacancies, the lookup tables
    const int slab_words = zl * D.L[1] * D.row_words * 3;
    const int64_t slab_off = D.occ_word_off + (int64_t)zb * D.L[1] * D.row_words * 3;
    for (int k = tid; k < slab_words; k += NT) S.occ[k] = occ[slab_off + k];
    for (int k = tid; k < D.L[0] + D.L[1] + D.L[2]; k += NT) {
        const int d = k < D.L[0] ? 0 : (k < D.L[0] + D.L[1] ? 1 : 2);
        const int c = d == 0 ? k : (d == 1 ? k - D.L[0] : k - D.L[0] - D.L[1]);
        S.frag_of_c[k] = (uint16_t)frag_of(c, D.base[d], D.rem[d]);
    }
    for (int z = tid; z < D.L[2]; z += NT) {
        const int fz = frag_of(z, D.base[2], D.rem[2]);
        int c = 0;
        while (c + 1 < P.ncta && P.fz0[c + 1] <= fz) ++c;
        S.zmap[z] = (uint32_t)c | ((uint32_t)(z - sh.zbeg[c]) << 8) | ((uint32_t)(fz - P.fz0[c]) << 18);
    }
    for (int lf = tid; lf < nfl_me; lf += NT) {
        const int fid = (fzb * D.nf[1]) * D.nf[0] + lf;  // layers are contiguous in the global order
        const int64_t g = D.frag_base + fid;
        const int c = counts[g];
        int head = -1;
        for (int k = 0; k < c && k < cap; ++k) {
            const int v = atomicAdd(&sh.pool_n, 1);
            if (v >= P.vcap) {
                atomicOr(status, STATUS_OVERFLOW);
                break;
            }
            const VacRec rr = recs[g * cap + k];
            int t, x, y, z;
            split_key(rr.key, t, x, y, z);
            S.key[v] = key32(t, x, y, z);
            S.d[3 * v] = rr.d[0];
            S.d[3 * v + 1] = rr.d[1];
            S.d[3 * v + 2] = rr.d[2];
            S.id[v] = rr.id;
            S.next[v] = (int16_t)head;
            head = v;
        }
        if (c > cap) atomicOr(status, STATUS_OVERFLOW);
        S.head[lf] = head;
        S.dirty[lf] = sh.cached ? rc.dirty[g] : 1;
        S.S[lf] = sh.cached ? rc.tot[g] : 0ull;
    }
    __syncthreads();
    {
        const int used = min(sh.pool_n, P.vcap);
        for (int k = tid; k < P.vcap - used; k += NT) S.fstack[k] = (int16_t)(used + k);
        if (tid == 0) sh.free_top = P.vcap - used;
    }
    cluster_sync();  // every slab is in place before any CTA reads a peer's

    const uint64_t hop_k1 = key_word(D.replica, PURPOSE_HOP);
    const int lane = tid & 31;
    const int warp = tid >> 5;
    const unsigned FULL = 0xffffffffu;
    int16_t* wslot = S.wslot + warp * cap;
    int8_t* wtype = S.wtype + warp * cap * 8;
    unsigned long long my_hops = 0, my_hand = 0;

    // the inbox of phase parity b into free slots and onto the fragments' lists
    auto drain = [&](int b) {
        const int n = min(sh.inbox_n[b], P.icap);
        if (sh.inbox_n[b] > P.icap && tid == 0) atomicOr(status, STATUS_OVERFLOW);
        for (int e = tid; e < n; e += NT) {
            const InboxRec r = S.inbox[b * P.icap + e];
            const int top = atomicSub(&sh.free_top, 1) - 1;
            if (top < 0) {
                atomicOr(status, STATUS_OVERFLOW);
                continue;
            }
            const int v = S.fstack[top];
            S.key[v] = r.key;
            S.d[3 * v] = r.d[0];
            S.d[3 * v + 1] = r.d[1];
            S.d[3 * v + 2] = r.d[2];
            S.id[v] = r.id;
            S.next[v] = (int16_t)atomicExch(S.head + r.lf, v);
            S.dirty[r.lf] = 1;
        }
        __syncthreads();
        if (tid == 0) {
            sh.inbox_n[b] = 0;
            if (sh.free_top < 0) sh.free_top = 0;
        }
    };

    // this slab's fragments of a colour: count per dimension, parity bits, first
    // fragment layer; and the coordinates of the colour's local fragment l
    auto colour_geo = [&](int colour, int cnt[2], int bit[3], int& lz0) -> int {
#pragma unroll
        for (int d = 0; d < 3; ++d) bit[d] = (colour >> d) & 1;
#pragma unroll
        for (int d = 0; d < 2; ++d) cnt[d] = D.nf[d] == 1 ? (bit[d] == 0 ? 1 : 0) : D.nf[d] / 2;
        lz0 = D.nf[2] == 1 ? 0 : (fzb + ((fzb & 1) != bit[2] ? 1 : 0));
        const int nlz = D.nf[2] == 1 ? (bit[2] == 0 ? 1 : 0) : (fze > lz0 ? (fze - lz0 + 1) / 2 : 0);
        return cnt[0] * cnt[1] * nlz;
    };
    auto frag_coords = [&](int l, const int cnt[2], const int bit[3], int lz0, int& f0, int& f1, int& f2) {
        f0 = l % cnt[0];
        f1 = (l / cnt[0]) % cnt[1];
        f2 = l / (cnt[0] * cnt[1]);
        f0 = D.nf[0] == 1 ? 0 : 2 * f0 + bit[0];
        f1 = D.nf[1] == 1 ? 0 : 2 * f1 + bit[1];
        f2 = lz0 + 2 * f2;
    };
    bool pre_valid = false;  // the phase's first draws were computed at the end of the last one

    uint32_t ph = 0;
    for (uint64_t wk = 0; wk < windows; ++wk) {
        const uint64_t w = D.window + wk;
        if ((wk & 63) == 0) {
            if (tid < 64 && wk + tid < windows) sh.perms[tid] = colour_perm_packed(D.seed, D.replica, w + tid);
            __syncthreads();
        }
        const uint32_t wperm = sh.perms[wk & 63];
        for (int p = 0; p < 8; ++p, ++ph) {
            if (ph > 0) drain((ph - 1) & 1);
            const int colour = (int)((wperm >> (4 * p)) & 15u);
            int cnt[2], bit[3], lz0;
            const int ncls = colour_geo(colour, cnt, bit, lz0);
            if (tid == 0) {
                sh.nact = 0;
                sh.next_act = 0;
            }
            __syncthreads();
            // ---- screen: one thread per local fragment of the colour
            for (int l = tid; l < ncls; l += NT) {
                int f0, f1, f2;
                frag_coords(l, cnt, bit, lz0, f0, f1, f2);
                const int lf = ((f2 - fzb) * D.nf[1] + f1) * D.nf[0] + f0;
                const int fid = (f2 * D.nf[1] + f1) * D.nf[0] + f0;
                if (S.head[lf] < 0) continue;
                const bool dirty = S.dirty[lf] != 0;
                const unsigned long long tot = S.S[lf];
                if (!dirty && tot == 0ull) continue;
                float E0, E1 = 0.f;
                uint64_t xs0, xs1;
                U64x4 blk{};
                if (pre_valid) {
                    E0 = S.pre_E[2 * l];
                    E1 = S.pre_E[2 * l + 1];
                    xs0 = S.pre_xs[2 * l];
                    xs1 = S.pre_xs[2 * l + 1];
                } else {
                    blk = philox4x64((uint64_t)fid, w, 0, 0, D.seed, hop_k1);
                    E0 = neglog32(blk.x[0]);
                    xs0 = blk.x[1];
                    xs1 = blk.x[3];
                }
                bool active = dirty;
                if (!active) {
                    const float ratio = __fdiv_rn(E0, __ull2float_rn(tot));
                    active = !(ratio > geo.theta_f);  // 0 + 2^F ratio <= theta
                }
                if (active) {
                    const int a = atomicAdd(&sh.nact, 1);
                    S.act[a] = f0 | (f1 << 10) | (f2 << 20);  // fragment coordinates (< 1024 each)
                    S.act_E[2 * a] = E0;
                    S.act_E[2 * a + 1] = pre_valid ? E1 : neglog32(blk.x[2]);
                    S.act_xs[2 * a] = xs0;
                    S.act_xs[2 * a + 1] = xs1;
                }
            }
            __syncthreads();
            // ---- run: one warp per listed fragment
            const int nact = sh.nact;
            for (;;) {
                int a = 0;
                if (lane == 0) a = atomicAdd(&sh.next_act, 1);
                a = __shfl_sync(FULL, a, 0);
                if (a >= nact) break;
                const int fxyz = S.act[a];
                const int fx = fxyz & 1023, fy = (fxyz >> 10) & 1023, fz = fxyz >> 20;
                const int lf = ((fz - fzb) * D.nf[1] + fy) * D.nf[0] + fx;
                const int fid = (fz * D.nf[1] + fy) * D.nf[0] + fx;
                const int lo0 = frag_start(fx, D.base[0], D.rem[0]), hi0 = frag_start(fx + 1, D.base[0], D.rem[0]);
                const int lo1 = frag_start(fy, D.base[1], D.rem[1]), hi1 = frag_start(fy + 1, D.base[1], D.rem[1]);
                const int lo2 = frag_start(fz, D.base[2], D.rem[2]), hi2 = frag_start(fz + 1, D.base[2], D.rem[2]);
                // slots: the fragment's vacancies in ascending site order
                int n = 0;
                if (lane == 0) {
                    for (int v = S.head[lf]; v >= 0; v = S.next[v]) {
                        if (n >= cap) {
                            atomicOr(status, STATUS_OVERFLOW);
                            break;
                        }
                        wslot[n++] = (int16_t)v;
                    }
                }
                n = __shfl_sync(FULL, n, 0);
                __syncwarp();
                // a list that received no vacancy since its last visit is still in site order
                bool ordered = false;
                uint32_t kk = 0xffffffffu;
                if (n <= 32) {  // rank by site (sites are distinct), unless already in order
                    const int vk = lane < n ? wslot[lane] : -1;
                    kk = lane < n ? S.key[vk] : 0xffffffffu;
                    const uint32_t kprev = __shfl_up_sync(FULL, kk, 1);
                    ordered = __ballot_sync(FULL, lane > 0 && lane < n && kprev > kk) == 0u;
                    if (!ordered) {
                        int rnk = 0;
                        for (int q = 0; q < n; ++q) rnk += __shfl_sync(FULL, kk, q) < kk ? 1 : 0;
                        __syncwarp();
                        if (lane < n) wslot[rnk] = (int16_t)vk;
                    }
                } else if (lane == 0) {
                    for (int k = 1; k < n; ++k) {
                        const int v = wslot[k];
                        const uint32_t kv = S.key[v];
                        int m = k;
                        while (m > 0 && S.key[wslot[m - 1]] > kv) {
                            wslot[m] = wslot[m - 1];
                            --m;
                        }
                        wslot[m] = (int16_t)v;
                    }
                }
                __syncwarp();
                const int nch = (n + 3) >> 2;
                // up to two chunks: each lane keeps its two slots' site keys in registers
                // (0xffffffff: no slot, or handed off), as in the replica-resident kernel
                uint32_t kc0 = 0xffffffffu, kc1 = 0xffffffffu;
                if (nch <= 2) {
                    const int m0 = lane >> 3, m1 = 4 + (lane >> 3);
                    if (ordered) {  // lane m holds slot m's key
                        const uint32_t a0 = __shfl_sync(FULL, kk, m0), a1 = __shfl_sync(FULL, kk, m1);
                        if (m0 < n) kc0 = a0;
                        if (m1 < n) kc1 = a1;
                    } else {
                        if (m0 < n) kc0 = S.key[wslot[m0]];
                        if (m1 < n) kc1 = S.key[wslot[m1]];
                    }
                }
                auto type_of = [&](uint32_t k, int q) -> int {
                    int t, x, y, z;
                    split32(k, t, x, y, z);
                    const NbEntry nbe = sh.nb[t][q];
                    const int code = csite_code(S, geo, me, nbe.t2, wrapc(x + nbe.dc[0], geo.L0),
                                                wrapc(y + nbe.dc[1], geo.L1), wrapc(z + nbe.dc[2], geo.L2));
                    return code == SP_V ? -1 : code * 3 + nbe.d[2] + 1;
                };
                int ty0 = -1, ty1 = -1;  // up to two chunks: rate types of events lane and 32 + lane
                auto compute_types = [&]() {
                    if (nch <= 2) {
                        ty0 = kc0 != 0xffffffffu ? type_of(kc0, lane & 7) : -1;
                        ty1 = (nch == 2 && kc1 != 0xffffffffu) ? type_of(kc1, lane & 7) : -1;
                    } else {
                        for (int c = 0; c < nch; ++c) {
                            const int e = c * 32 + lane, m = e >> 3;
                            int ty = -1;
                            if (m < n && wslot[m] >= 0) ty = type_of(S.key[wslot[m]], e & 7);
                            wtype[e] = (int8_t)ty;
                        }
                    }
                    __syncwarp();
                };
                compute_types();

                double clock = 0.0;
                uint64_t i = 0, batch = ~0ull;
                uint64_t xs_even = 0, xs_odd = 0;
                float E_even = 0.f, E_odd = 0.f;
                unsigned long long tot = 0;
                for (;;) {
                    // exact total (order-free integer sum) and, for up to two chunks, the
                    // inclusive prefixes the selection needs
                    unsigned long long inc0 = 0, inc1 = 0;
                    if (nch <= 2) {
                        const int t0 = ty0;
                        inc0 = t0 < 0 ? 0ull : (unsigned long long)D.q[t0];
#pragma unroll
                        for (int off = 1; off < 32; off <<= 1) {
                            const unsigned long long t2 = __shfl_up_sync(FULL, inc0, off);
                            if (lane >= off) inc0 += t2;
                        }
                        tot = __shfl_sync(FULL, inc0, 31);
                        if (nch == 2) {
                            const int t1 = ty1;
                            inc1 = t1 < 0 ? 0ull : (unsigned long long)D.q[t1];
#pragma unroll
                            for (int off = 1; off < 32; off <<= 1) {
                                const unsigned long long t2 = __shfl_up_sync(FULL, inc1, off);
                                if (lane >= off) inc1 += t2;
                            }
                            inc1 += tot;
                            tot = __shfl_sync(FULL, inc1, 31);
                        }
                    } else {
                        unsigned long long part = 0;
                        for (int c = 0; c < nch; ++c) {
                            const int ty = wtype[c * 32 + lane];
                            part += ty < 0 ? 0ull : (unsigned long long)D.q[ty];
                        }
#pragma unroll
                        for (int off = 16; off; off >>= 1) part += __shfl_xor_sync(FULL, part, off);
                        tot = part;
                    }
                    if (tot == 0ull) break;
                    if (i >= MAX_EVENTS_PER_PHASE) {
                        if (lane == 0) atomicOr(status, STATUS_EVENT_LIMIT);
                        break;
                    }
                    uint64_t xs;
                    float E;
                    if (i < 2) {
                        xs = S.act_xs[2 * a + (int)i];
                        E = S.act_E[2 * a + (int)i];
                    } else {
                        const uint64_t k = i - 2;
                        if ((k >> 6) != batch) {
                            batch = k >> 6;
                            const U64x4 blk =
                                philox4x64((uint64_t)fid, w, 1 + 32 * batch + lane, 0, D.seed, hop_k1);
                            xs_even = blk.x[1];
                            xs_odd = blk.x[3];
                            E_even = neglog32(blk.x[0]);
                            E_odd = neglog32(blk.x[2]);
                        }
                        const int src = (int)((k >> 1) & 31);
                        const bool odd = (k & 1) != 0;
                        xs = __shfl_sync(FULL, odd ? xs_odd : xs_even, src);
                        E = __shfl_sync(FULL, odd ? E_odd : E_even, src);
                    }
                    const float ratio = __fdiv_rn(E, __ull2float_rn(tot));
                    const double nclock = __dadd_rn(clock, scale_pow2((double)ratio, geo.F));
                    const bool past = i == 0 ? ratio > geo.theta_f : nclock > geo.theta;  // the first: clock 0
                    // up to two chunks: the selection (no side effects) before the clock test,
                    // so that its shuffles overlap the clock's FP64 chain; a break discards it
                    const unsigned long long target = __umul64hi(xs, tot);
                    int e_sel = -1;
                    uint32_t ksel = 0u;
                    int tsel = -1;
                    if (nch <= 2) {
                        unsigned bal = __ballot_sync(FULL, inc0 > target);
                        if (bal) {
                            e_sel = __ffs(bal) - 1;
                        } else {
                            bal = __ballot_sync(FULL, inc1 > target);
                            if (bal && nch == 2) e_sel = 32 + __ffs(bal) - 1;
                        }
                        const int ms = e_sel >> 3;  // the slot's site key and the event's type
                        ksel = __shfl_sync(FULL, ms < 4 ? kc0 : kc1, (ms & 3) << 3);
                        tsel = __shfl_sync(FULL, e_sel < 32 ? ty0 : ty1, e_sel & 31);
                    }
                    if (past) break;
                    if (nch > 2) {
                        unsigned long long carry = 0;
                        for (int c = 0; c < nch; ++c) {
                            const int ty = wtype[c * 32 + lane];
                            unsigned long long inc = ty < 0 ? 0ull : (unsigned long long)D.q[ty];
#pragma unroll
                            for (int off = 1; off < 32; off <<= 1) {
                                const unsigned long long t2 = __shfl_up_sync(FULL, inc, off);
                                if (lane >= off) inc += t2;
                            }
                            inc += carry;
                            const unsigned bal = __ballot_sync(FULL, inc > target);
                            if (bal) {
                                e_sel = c * 32 + __ffs(bal) - 1;
                                break;
                            }
                            carry = __shfl_sync(FULL, inc, 31);
                        }
                    }
                    if (e_sel < 0) {  // cannot happen: the target lies below the total
                        if (lane == 0) atomicOr(status, STATUS_OVERFLOW);
                        break;
                    }
                    const int m = e_sel >> 3, qd = e_sel & 7;
                    int t, x, y, z;
                    split32(nch <= 2 ? ksel : S.key[wslot[m]], t, x, y, z);
                    const NbEntry nb = sh.nb[t][qd];
                    const NbSite j = cnb_site(sh, geo, t, x, y, z, qd);
                    const bool owned = j.jx >= lo0 && j.jx < hi0 && j.jy >= lo1 && j.jy < hi1 && j.jz >= lo2 &&
                                       j.jz < hi2;
                    if (lane == 0) {  // apply the exchange
                        const int v = wslot[m];
                        const uint32_t ion = (uint32_t)((nch <= 2 ? tsel : (int)wtype[e_sel]) / 3);
                        csite_xor(S, geo, me, t, x, y, z, ((uint32_t)SP_V ^ ion) << occ_shift(x));
                        csite_xor(S, geo, me, j.t2, j.jx, j.jy, j.jz, (ion ^ (uint32_t)SP_V) << occ_shift(j.jx));
                        const int d0 = S.d[3 * v] + nb.d[0], d1 = S.d[3 * v + 1] + nb.d[1],
                                  d2 = S.d[3 * v + 2] + nb.d[2];
                        if (tracer) {
                            const int64_t s_lin = (((int64_t)t * D.L[2] + z) * D.L[1] + y) * D.L[0] + x;
                            const int64_t j_lin = (((int64_t)j.t2 * D.L[2] + j.jz) * D.L[1] + j.jy) * D.L[0] + j.jx;
                            int32_t* ts = tracer + 3 * (D.site_off + s_lin);
                            int32_t* tj = tracer + 3 * (D.site_off + j_lin);
                            ts[0] = tj[0] - nb.d[0];
                            ts[1] = tj[1] - nb.d[1];
                            ts[2] = tj[2] - nb.d[2];
                            tj[0] = tj[1] = tj[2] = 0;
                        }
                        const uint32_t jk = key32(j.t2, j.jx, j.jy, j.jz);
                        if (owned) {
                            S.d[3 * v] = d0;
                            S.d[3 * v + 1] = d1;
                            S.d[3 * v + 2] = d2;
                            S.key[v] = jk;
                        } else {
                            wslot[m] = -1;
                            uint32_t o2;
                            int lf2;
                            cowner(S, geo, j.jx, j.jy, j.jz, o2, lf2);
                            if (o2 == me) {  // another fragment of this slab: onto its list
                                S.d[3 * v] = d0;
                                S.d[3 * v + 1] = d1;
                                S.d[3 * v + 2] = d2;
                                S.key[v] = jk;
                                S.next[v] = (int16_t)atomicExch(S.head + lf2, v);
                            } else {  // another slab: into its inbox, the slot back to the free stack
                                const int bidx = (int)(ph & 1u);
                                const uint32_t e =
                                    atom_peer_add(peer_addr(&sh.inbox_n[bidx], o2), 1u);
                                if ((int)e < P.icap) {
                                    const uint32_t base = peer_addr(S.inbox + bidx * P.icap + (int)e, o2);
                                    st_peer(base, jk);
                                    st_peer(base + 4, d0);
                                    st_peer(base + 8, d1);
                                    st_peer(base + 12, d2);
                                    st_peer(base + 16, S.id[v]);
                                    st_peer(base + 20, lf2);
                                } else {
                                    atomicOr(status, STATUS_OVERFLOW);
                                }
                                S.fstack[atomicAdd(&sh.free_top, 1)] = (int16_t)v;
                            }
                            ++my_hand;
                        }
                    }
                    __syncwarp();
                    if (nch <= 2) {  // the moved vacancy's lanes follow it (or drop a handed-off slot)
                        const uint32_t nk = owned ? key32(j.t2, j.jx, j.jy, j.jz) : 0xffffffffu;
                        if ((lane >> 3) == m) kc0 = nk;
                        if (4 + (lane >> 3) == m) kc1 = nk;
                    }
                    {
                        // the fragments whose totals changed: owners of the vacancies next to the
                        // two changed sites (lanes 0-7 look around s, 8-15 around j; 16-31 repeat
                        // them without storing, so that no branch splits the warp)
                        const int pl = lane & 15;
                        const int bt = pl < 8 ? t : j.t2;
                        const int bx = pl < 8 ? x : j.jx, by = pl < 8 ? y : j.jy, bz = pl < 8 ? z : j.jz;
                        const NbSite c = cnb_site(sh, geo, bt, bx, by, bz, pl & 7);
                        const bool vac = csite_code(S, geo, me, c.t2, c.jx, c.jy, c.jz) == SP_V;
                        uint32_t oc;
                        int lc;
                        cowner(S, geo, c.jx, c.jy, c.jz, oc, lc);
                        compute_types();
                        if (lane < 16 && vac) {
                            if (oc == me) {
                                if (lc != lf) S.dirty[lc] = 1;
                            } else {
                                st_peer8(peer_addr(S.dirty + lc, oc), 1);
                            }
                        }
                    }
                    clock = nclock;
                    ++i;
                }
                // surviving vacancies stay linked to this fragment, in slot order (up to 32
                // slots, each lane links its own slot to the next live one)
                int head = -1;
                if (n <= 32) {
                    const int v = lane < n ? wslot[lane] : -1;
                    const unsigned live = __ballot_sync(FULL, v >= 0);
                    const unsigned later = live & ~((2u << lane) - 1u);
                    const int vn = __shfl_sync(FULL, v, later ? __ffs(later) - 1 : 0);
                    const int hv = __shfl_sync(FULL, v, live ? __ffs(live) - 1 : 0);
                    if (v >= 0) S.next[v] = (int16_t)(later ? vn : -1);
                    head = live ? hv : -1;
                }
                if (lane == 0) {
                    if (n > 32) {
                        for (int m = n - 1; m >= 0; --m) {
                            const int v = wslot[m];
                            if (v < 0) continue;
                            S.next[v] = (int16_t)head;
                            head = v;
                        }
                    }
                    S.head[lf] = head;
                    S.S[lf] = tot;
                    S.dirty[lf] = 0;
                    my_hops += i;
                }
                __syncwarp();
            }
            // every write of the phase, local and remote, is visible after the wait.
            // Between arrival and wait: the next phase's first draws (events 0 and 1
            // of each of this CTA's fragments of the next colour), which depend on no
            // fragment's state, so that they overlap the barrier's release
            cluster_arrive();
            pre_valid = false;
            {
                int ncolour = -1;
                uint64_t nw = w;
                if (p < 7) {
                    ncolour = (int)((wperm >> (4 * (p + 1))) & 15u);
                } else if (wk + 1 < windows && ((wk + 1) & 63) != 0) {  // the next window's order is known
                    ncolour = (int)(sh.perms[(wk + 1) & 63] & 15u);
                    nw = w + 1;
                }
                if (ncolour >= 0) {
                    int ncnt[2], nbit[3], nlz0;
                    const int nn = colour_geo(ncolour, ncnt, nbit, nlz0);
                    for (int l = tid; l < nn; l += NT) {
                        int f0, f1, f2;
                        frag_coords(l, ncnt, nbit, nlz0, f0, f1, f2);
                        const int fid = (f2 * D.nf[1] + f1) * D.nf[0] + f0;
                        const U64x4 blk = philox4x64((uint64_t)fid, nw, 0, 0, D.seed, hop_k1);
                        S.pre_E[2 * l] = neglog32(blk.x[0]);
                        S.pre_E[2 * l + 1] = neglog32(blk.x[2]);
                        S.pre_xs[2 * l] = blk.x[1];
                        S.pre_xs[2 * l + 1] = blk.x[3];
                    }
                    pre_valid = true;
                }
            }
            __syncwarp();
            cluster_wait();
        }
    }
    if (ph > 0) drain((ph - 1) & 1);

    // ---- stage out: this slab's occupancy, its fragments' records
    for (int k = tid; k < slab_words; k += NT) occ[slab_off + k] = S.occ[k];
    for (int lf = tid; lf < nfl_me; lf += NT) {
        const int64_t g = D.frag_base + (int64_t)fzb * D.nf[1] * D.nf[0] + lf;
        int k = 0;
        for (int v = S.head[lf]; v >= 0; v = S.next[v], ++k) {
            if (k >= cap) {
                atomicOr(status, STATUS_OVERFLOW);
                break;
            }
            int t, x, y, z;
            split32(S.key[v], t, x, y, z);
            VacRec rr;
            rr.key = make_key(t, x, y, z);
            rr.d[0] = S.d[3 * v];
            rr.d[1] = S.d[3 * v + 1];
            rr.d[2] = S.d[3 * v + 2];
            rr.id = S.id[v];
            recs[g * cap + k] = rr;
        }
        counts[g] = k;
        rc.tot[g] = S.S[lf];
        rc.dirty[g] = S.dirty[lf];
    }
    atomicAdd(&sh.hops, my_hops);
    atomicAdd(&sh.hand, my_hand);
    __syncthreads();
    if (tid == 0) {
        if (sh.hops) atomicAdd(stats + 2 * P.rep, sh.hops);
        if (sh.hand) atomicAdd(stats + 2 * P.rep + 1, sh.hand);
    }
    cluster_sync();  // no CTA leaves while a peer may still address it
    if (tid == 0 && me == 0) rc.valid[P.rep] = 1;
}

size_t cluster_smem_bytes(const RepDesc& D, const ClusterPlan& p, int cap)
{
    return cluster_layout_bytes(D, p, cap, CLUSTER_THREADS / 32, nullptr);
}

bool make_cluster_plan(const RepDesc& D, int64_t n_vac, int cap, int min_ctas, int max_ctas, ClusterPlan* out)
{
    if (D.L[0] > 1024 || D.L[1] > 1024 || D.L[2] > 1024 || D.nf[2] < 2) return false;
    const int nf2 = D.nf[2];
    for (int nc = std::max(2, min_ctas); nc <= std::min(max_ctas, CLUSTER_MAX_CTAS) && nc <= nf2; ++nc) {
        ClusterPlan p{};
        p.ncta = nc;
        int zs = 0, layers = 0;
        for (int c = 0; c <= nc; ++c) p.fz0[c] = (int)((int64_t)c * nf2 / nc);
        for (int c = 0; c < nc; ++c) {
            const int z0 = p.fz0[c] * D.base[2] + std::min(p.fz0[c], D.rem[2]);
            const int z1 = p.fz0[c + 1] * D.base[2] + std::min(p.fz0[c + 1], D.rem[2]);
            zs = std::max(zs, z1 - z0);
            layers = std::max(layers, p.fz0[c + 1] - p.fz0[c]);
        }
        p.zs = zs;
        p.nfl = layers * D.nf[0] * D.nf[1];
        // the inbox takes a phase's arrivals through the slab's two faces: at most the
        // vacancies of the two neighbouring cell layers (a vacancy crosses once per
        // phase), with a margin of eight standard deviations
        const double per_layer = 2.0 * (double)n_vac / D.L[2];
        p.icap = (int)std::min<double>(8192.0, std::ceil(per_layer + 8.0 * std::sqrt(per_layer) + 64.0));
        // the vacancy pool: whatever shared memory is left, at least twice the slab's share
        p.vcap = 0;
        const size_t fixed = cluster_layout_bytes(D, p, cap, CLUSTER_THREADS / 32, nullptr);
        if (fixed > RESIDENT_MAX_SMEM) continue;
        const int64_t share = (n_vac * layers + nf2 - 1) / nf2;
        const int64_t room = (int64_t)(RESIDENT_MAX_SMEM - fixed) / 24 - 64;
        const int64_t vcap = std::min<int64_t>(32767, room);
        if (vcap < 2 * share + 64) continue;
        p.vcap = (int)vcap;
        if (cluster_layout_bytes(D, p, cap, CLUSTER_THREADS / 32, nullptr) > RESIDENT_MAX_SMEM) continue;
        *out = p;
        return true;
    }
    return false;
}

cudaError_t cluster_prepare()
{
    cudaError_t e = cudaFuncSetAttribute(k_cluster<CLUSTER_THREADS>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)RESIDENT_MAX_SMEM);
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(k_cluster<CLUSTER_THREADS>, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
    return e;
}

int cluster_fits(int ncta, size_t smem)
{
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3((unsigned)ncta);
    cfg.blockDim = dim3(CLUSTER_THREADS);
    cfg.dynamicSmemBytes = smem;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = (unsigned)ncta;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    int n = 0;
    if (cudaOccupancyMaxActiveClusters(&n, k_cluster<CLUSTER_THREADS>, &cfg) != cudaSuccess) {
        cudaGetLastError();
        return 0;
    }
    return n;
}

cudaError_t launch_cluster(const RepDesc* d_descs, const ClusterPlan* d_plans, int nplans, int ncta, size_t smem,
                           uint64_t windows, uint32_t* occ, VacRec* recs, int32_t* counts, int32_t* tracer,
                           unsigned long long* stats, uint32_t* status, int cap, const NbTable& nbt,
                           const ResCache& rc, cudaStream_t st)
{
    if (nplans <= 0) return cudaSuccess;
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3((unsigned)(ncta * nplans));
    cfg.blockDim = dim3(CLUSTER_THREADS);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = st;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = (unsigned)ncta;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, k_cluster<CLUSTER_THREADS>, d_descs, d_plans, windows, occ, recs, counts, tracer,
                              stats, status, cap, nbt, rc);
}

cudaError_t resident_prepare()
{
    cudaError_t e = cudaSuccess;
    for (auto fn : {k_resident<128, 1>, k_resident<256, 1>, k_resident<512, 1>, k_resident<1024, 1>,
                    k_resident<1024, 2>}) {
        e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)RESIDENT_MAX_SMEM);
        if (e != cudaSuccess) return e;
    }
    return e;
}

cudaError_t launch_resident(const RepDesc* d_descs, const int32_t* d_reps, int nreps, const int64_t* d_nvac,
                            size_t smem, int threads, int cluster, uint64_t windows, uint32_t* occ, VacRec* recs,
                            int32_t* counts, int32_t* tracer, unsigned long long* stats, uint32_t* status,
                            int cap, const NbTable& nbt, uint32_t stuck_wait_us, const ResCache& rc, cudaStream_t st)
{
    if (nreps <= 0) return cudaSuccess;
    if (cluster == 2 && threads == 1024) {
        cudaLaunchConfig_t cfg = {};
        cfg.gridDim = dim3(2u * nreps);
        cfg.blockDim = dim3(1024);
        cfg.dynamicSmemBytes = smem;
        cfg.stream = st;
        cudaLaunchAttribute attr[1];
        attr[0].id = cudaLaunchAttributeClusterDimension;
        attr[0].val.clusterDim.x = 2;
        attr[0].val.clusterDim.y = 1;
        attr[0].val.clusterDim.z = 1;
        cfg.attrs = attr;
        cfg.numAttrs = 1;
        return cudaLaunchKernelEx(&cfg, k_resident<1024, 2>, d_descs, d_reps, d_nvac, windows, occ, recs, counts,
                                  tracer, stats, status, cap, nbt, stuck_wait_us, rc);
    }
    if (threads == 128)
        k_resident<128, 1><<<nreps, 128, smem, st>>>(d_descs, d_reps, d_nvac, windows, occ, recs, counts, tracer,
                                                     stats, status, cap, nbt, stuck_wait_us, rc);
    else if (threads == 256)
        k_resident<256, 1><<<nreps, 256, smem, st>>>(d_descs, d_reps, d_nvac, windows, occ, recs, counts, tracer,
                                                     stats, status, cap, nbt, stuck_wait_us, rc);
    else if (threads == 1024)
        k_resident<1024, 1><<<nreps, 1024, smem, st>>>(d_descs, d_reps, d_nvac, windows, occ, recs, counts,
                                                       tracer, stats, status, cap, nbt, stuck_wait_us, rc);
    else
        k_resident<512, 1><<<nreps, 512, smem, st>>>(d_descs, d_reps, d_nvac, windows, occ, recs, counts, tracer,
                                                     stats, status, cap, nbt, stuck_wait_us, rc);
    return cudaGetLastError();
}

}  // namespace fkmc
