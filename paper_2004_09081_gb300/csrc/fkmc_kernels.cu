// fkmc_kernels.cu -- sm_103a kernels of the fragment kMC library.
//
//   k_init       placement of vacancies and H- (keyed Feistel bijection)
//   k_phase      one colour phase: every fragment of the phase's colour runs
//                BKL on its own vacancies until its next event would pass the
//                window length (arXiv:2004.09081 Sec. II.A Eqs. RateCnst1,
//                eventSelection, TimeStep; fragment-local selection Sec. II.B
//                Eq. AtomP).  One warp per fragment.
//   k_moments_*  exact integer displacement moments (Sec. III: D from tracked
//                trajectories).
//   k_field_*    site energies of the dopant/defect section: the energy field
//                E_site of every O site, scattered from vacancies and dopants.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstring>

#include "fkmc_device.cuh"
#include "fkmc_kernels.h"

namespace fkmc {

__constant__ NbEntry c_nb[3][8];
// The same table in global memory for lookups whose (t, n) differ across the
// lanes of a warp: a global load serves them in one or two L1 wavefronts, a
// constant-memory load would be split into one request per distinct entry.
__device__ __align__(8) NbEntry g_nb[3][8];

__device__ __forceinline__ NbEntry nb_entry(int t, int n)
{
    const uint2 v = __ldg(reinterpret_cast<const uint2*>(&g_nb[0][0]) + 8 * t + n);
    NbEntry e;
    memcpy(&e, &v, sizeof e);
    return e;
}

// ------------------------------------------------------------------ init
__global__ void k_init(RepDesc D, int b_bits, int64_t n_vac, int64_t n_total, uint32_t* occ,
                       VacRec* recs, int32_t* counts, int cap, uint32_t* status)
{
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n_total) return;
    const uint64_t mask = (1ull << b_bits) - 1ull;
    const uint64_t k0 = D.seed, k1 = key_word(D.replica, PURPOSE_INIT);
    uint64_t v = (uint64_t)i;
    do {
        uint64_t Lh = v >> b_bits, Rh = v & mask;
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            const U64x4 o = philox4x64(Rh, (uint64_t)k, 0, 0, k0, k1);
            const uint64_t nr = Lh ^ (o.x[0] & mask);
            Lh = Rh;
            Rh = nr;
        }
        v = (Lh << b_bits) | Rh;
    } while (v >= (uint64_t)D.nsite);
    const int x = (int)(v % D.L[0]);
    const int y = (int)((v / D.L[0]) % D.L[1]);
    const int z = (int)((v / ((uint64_t)D.L[0] * D.L[1])) % D.L[2]);
    const int t = (int)(v / ((uint64_t)D.L[0] * D.L[1] * D.L[2]));
    const uint32_t code = i < n_vac ? (uint32_t)SP_V : (uint32_t)SP_H;
    atomicOr(occ + occ_word(D, t, x, y, z), code << occ_shift(x));
    if (i < n_vac) {
        const int fx = frag_of(x, D.base[0], D.rem[0]);
        const int fy = frag_of(y, D.base[1], D.rem[1]);
        const int fz = frag_of(z, D.base[2], D.rem[2]);
        const int64_t g = D.frag_base + ((int64_t)fz * D.nf[1] + fy) * D.nf[0] + fx;
        const int slot = atomicAdd(counts + g, 1);
        if (slot < cap) {
            VacRec r;
            r.key = make_key(t, x, y, z);
            r.d[0] = r.d[1] = r.d[2] = 0;
            r.id = (uint32_t)i;
            recs[g * cap + slot] = r;
        } else {
            atomicOr(status, STATUS_OVERFLOW);
        }
    }
}

// ------------------------------------------------------------------ phase
template <int PREC>
struct Arith;

// FP64 plain form: rates are doubles, prefix sums in the canonical order.
template <>
struct Arith<0> {
    using V = double;
    static __device__ __forceinline__ V zero() { return 0.0; }
    static __device__ __forceinline__ V add(V a, V b) { return __dadd_rn(a, b); }
    template <bool GRAIN = false>
    static __device__ __forceinline__ V rate(const RepDesc& D, int ty)
    {
        if constexpr (GRAIN) return ty < 0 ? 0.0 : (ty < 6 ? D.k64[ty] : D.k64g[ty - 6]);
        else return ty < 0 ? 0.0 : D.k64[ty];
    }
    static __device__ __forceinline__ V shfl_up(V v, int off) { return __shfl_up_sync(0xffffffffu, v, off); }
    static __device__ __forceinline__ V shfl(V v, int src) { return __shfl_sync(0xffffffffu, v, src); }
    static __device__ __forceinline__ bool pos(V v) { return v > 0.0; }
};

// Mixed form: u64 fixed-point rates, exact integer sums.
template <>
struct Arith<1> {
    using V = unsigned long long;
    static __device__ __forceinline__ V zero() { return 0ull; }
    static __device__ __forceinline__ V add(V a, V b) { return a + b; }
    template <bool GRAIN = false>
    static __device__ __forceinline__ V rate(const RepDesc& D, int ty)
    {
        if constexpr (GRAIN) return ty < 0 ? 0ull : (V)(ty < 6 ? D.q[ty] : D.qg[ty - 6]);
        else return ty < 0 ? 0ull : (V)D.q[ty];
    }
    static __device__ __forceinline__ V shfl_up(V v, int off) { return __shfl_up_sync(0xffffffffu, v, off); }
    static __device__ __forceinline__ V shfl(V v, int src) { return __shfl_sync(0xffffffffu, v, src); }
    static __device__ __forceinline__ bool pos(V v) { return v != 0ull; }
};

// Inclusive Kogge-Stone scan over the 32 lanes (strides 1,2,4,8,16), the
// canonical order of the plain form's partial sums.
template <int PREC>
__device__ __forceinline__ typename Arith<PREC>::V warp_scan(typename Arith<PREC>::V v, int lane)
{
    using A = Arith<PREC>;
#pragma unroll
    for (int off = 1; off < 32; off <<= 1) {
        const typename A::V t = A::shfl_up(v, off);
        if (lane >= off) v = A::add(v, t);
    }
    return v;
}

struct WarpSmem {
    VacRec* rec;     // [cap] records as loaded (slot data lives here)
    uint16_t* order; // [cap] slot m -> index into rec
    int8_t* types;   // [8*cap] rate type of event e, -1 = no event
    uint8_t* alive;  // [cap]
    double* rate;    // [8*cap] FP64 rate of event e (site-energy path only)
};

__host__ __device__ inline size_t warp_rate_offset(int cap) { return (size_t)((35 * cap + 7) / 8) * 8; }

__device__ __forceinline__ WarpSmem carve(unsigned char* base, int cap)
{
    WarpSmem s;
    s.rec = reinterpret_cast<VacRec*>(base);
    s.order = reinterpret_cast<uint16_t*>(base + 24 * cap);
    s.types = reinterpret_cast<int8_t*>(base + 26 * cap);
    s.alive = reinterpret_cast<uint8_t*>(base + 34 * cap);
    s.rate = reinterpret_cast<double*>(base + warp_rate_offset(cap));
    return s;
}

// Per-warp shared memory in bytes.  Kept in 32-bit arithmetic (cap <= 256):
// the run pass multiplies it by the warp index for its base address, and a
// 64-bit product there costs the kernel registers it cannot spare.
__host__ __device__ inline size_t warp_smem_bytes(int cap, bool site)
{
    const int b = site ? (35 * cap + 7) / 8 * 8 + 64 * cap : 35 * cap;
    return (size_t)((b + 15) / 16) * 16;
}

// Rate types of every event of the fragment, read from the occupancy words
// in L2 (ld.global.cg, so that this warp's own exchanges are seen).
template <bool GRAIN = false>
__device__ __forceinline__ void compute_types(const RepDesc& D, const uint32_t* occ, const WarpSmem& S,
                                              int nslots, int nch, int lane, const uint8_t* gb = nullptr)
{
    for (int c = 0; c < nch; ++c) {
        const int e = c * 32 + lane;
        const int m = e >> 3, n = e & 7;
        int ty = -1;
        if (m < nslots && S.alive[m]) {
            int t, x, y, z;
            split_key(S.rec[S.order[m]].key, t, x, y, z);
            const NbEntry nb = nb_entry(t, n);
            const int jx = wrapc(x + nb.dc[0], D.L[0]);
            const int jy = wrapc(y + nb.dc[1], D.L[1]);
            const int jz = wrapc(z + nb.dc[2], D.L[2]);
            const uint32_t w = __ldcg(occ + occ_word(D, nb.t2, jx, jy, jz));
            const int code = (int)((w >> occ_shift(jx)) & 3u);
            ty = code == SP_V ? -1 : code * 3 + nb.d[2] + 1;
            if constexpr (GRAIN) {  // a hop touching a boundary cell takes the raised table
                if (ty >= 0 && (gb[cell_index(D, x, y, z)] | gb[cell_index(D, jx, jy, jz)])) ty += 6;
            }
        }
        S.types[e] = (int8_t)ty;
    }
}

__device__ __forceinline__ int64_t site_lin(const RepDesc& D, int t, int x, int y, int z)
{
    return (((int64_t)t * D.L[2] + z) * D.L[1] + y) * D.L[0] + x;
}

// Site-energy path: rate type and FP64 rate of every event (type + 6 for a
// hop touching a grain-boundary cell, whose table rate is the raised one).  The barrier of
// the hop s -> j is Ea + dU/2 + (E_site(j) - E_site(s))/2, E_site(j) without the
// hopping vacancy itself (which sits in j's a/sqrt2 shell); the energy
// difference m (1e-4 eV units) enters as k_table * hi[m >> 9] * lo[m & 511],
// two FP64 products in that order.  Field words are read from L2 (ld.cg):
// other warps of the phase update them with atomics.
template <bool GRAIN>
__device__ __forceinline__ void compute_rates_site(const RepDesc& D, const uint32_t* occ, const SiteArgs& sa,
                                                   const WarpSmem& S, int nslots, int nch, int lane,
                                                   uint32_t* status)
{
    const double* lo = sa.btab + D.btab_off;
    const double* hi = lo + BOLTZ_LO;
    const int32_t* field = sa.field + D.site_off;
    for (int c = 0; c < nch; ++c) {
        const int e = c * 32 + lane;
        const int m = e >> 3, n = e & 7;
        int ty = -1;
        double k = 0.0;
        if (m < nslots && S.alive[m]) {
            int t, x, y, z;
            split_key(S.rec[S.order[m]].key, t, x, y, z);
            const NbEntry nb = nb_entry(t, n);
            const int jx = wrapc(x + nb.dc[0], D.L[0]);
            const int jy = wrapc(y + nb.dc[1], D.L[1]);
            const int jz = wrapc(z + nb.dc[2], D.L[2]);
            const uint32_t w = __ldcg(occ + occ_word(D, nb.t2, jx, jy, jz));
            const int code = (int)((w >> occ_shift(jx)) & 3u);
            if (code != SP_V) {
                ty = code * 3 + nb.d[2] + 1;
                double k0 = D.k64[ty];
                if constexpr (GRAIN) {
                    if (sa.gbound[cell_index(D, x, y, z)] | sa.gbound[cell_index(D, jx, jy, jz)]) {
                        k0 = D.k64g[ty];
                        ty += 6;
                    }
                }
                const int32_t Es = __ldcg(field + site_lin(D, t, x, y, z));
                const int32_t Ej = __ldcg(field + site_lin(D, nb.t2, jx, jy, jz));
                int32_t dm = Ej - sa.e_self - Es;
                if (sa.g_elec) dm -= sa.g_elec[24 * D.replica + 8 * t + n];
                const int hidx = D.bhi_mid + (dm >> 9);
                if (hidx >= 0 && hidx < D.bhi_len) {
                    k = __dmul_rn(__dmul_rn(k0, __ldg(hi + hidx)), __ldg(lo + (dm & 511)));
                } else {  // outside the bound the tables were built for: report, no event
                    atomicOr(status, STATUS_ENERGY_RANGE);
                    ty = -1;
                }
            }
        }
        S.types[e] = (int8_t)ty;
        S.rate[e] = k;
    }
}

// Move the hopping vacancy's share of the energy field from s to j: every O
// site in a V-V shell of s loses the shell energy, every one around j gains it.
// Integer atomics: fragments of one colour may touch the same field word.
__device__ __forceinline__ void move_field(const RepDesc& D, const SiteArgs& sa, int t, int x, int y, int z, int t2,
                                           int jx, int jy, int jz, int lane)
{
    int32_t* field = sa.field + D.site_off;
    for (int o = lane; o < sa.n_vv; o += 32) {
        const SiteOff a = sa.vv[t * SITE_MAX_VV + o];
        atomicAdd(field + site_lin(D, a.t2, wrapc(x + a.dc[0], D.L[0]), wrapc(y + a.dc[1], D.L[1]),
                                   wrapc(z + a.dc[2], D.L[2])),
                  -a.e);
        const SiteOff b = sa.vv[t2 * SITE_MAX_VV + o];
        atomicAdd(field + site_lin(D, b.t2, wrapc(jx + b.dc[0], D.L[0]), wrapc(jy + b.dc[1], D.L[1]),
                                   wrapc(jz + b.dc[2], D.L[2])),
                  b.e);
    }
}

// Coordinates (c0, c1, c2) of index i in an n0 x n1 x n2 box, i = (c2 n1 + c1) n0 + c0:
// 32-bit division where the index fits (a 64-bit division is a long
// instruction sequence on the GPU).
__device__ __forceinline__ void unflatten3(int64_t i, int n0, int n1, int c[3])
{
    if (i <= 0x7fffffffll) {
        const unsigned u = (unsigned)i, m0 = (unsigned)n0, m1 = (unsigned)n1;
        const unsigned q = u / m0;
        c[0] = (int)(u - q * m0);
        c[1] = (int)(q % m1);
        c[2] = (int)(q / m1);
    } else {
        c[0] = (int)(i % n0);
        c[1] = (int)((i / n0) % n1);
        c[2] = (int)(i / ((int64_t)n0 * n1));
    }
}

// Per-window set-up: colour order of every replica for this window, and the
// counters of the 8 phases cleared (act_count: 3 lists x 8 phases, then the
// one-thread-per-fragment pass's window tickets of each phase).  wctl[0] counts the windows of the
// current kmc_run call, wctl[1] holds the offset of the window being run.
// Every block reads wctl[0] here, so it is advanced later, by the first
// screen pass of the window (a later launch on the same stream).
__global__ void k_window_setup(const RepDesc* __restrict__ descs, int nrep, unsigned long long* wctl,
                               uint32_t* perms, int32_t* act_count)
{
    const uint64_t wk = wctl[0];
    for (int r = blockIdx.x * blockDim.x + threadIdx.x; r < nrep; r += gridDim.x * blockDim.x)
        perms[r] = colour_perm_packed(descs[r].seed, descs[r].replica, descs[r].window + wk);
    if (blockIdx.x == 0 && threadIdx.x < ACT_COUNTERS) act_count[threadIdx.x] = 0;
    if (blockIdx.x == 0 && threadIdx.x == 0) wctl[1] = wk;
}

// Fragment of work item `item` in colour phase `phase`: the replica (binary
// search over the items' prefix) and the fragment index inside it, or false
// where the replica has fewer fragments of that colour than items or runs in
// the replica-resident kernel.  Each replica's items enumerate the fragments
// of one colour (parity bits per dimension; a single-fragment dimension holds
// only colour bit 0).
__device__ __forceinline__ bool item_fragment(const RepDesc* __restrict__ descs, int nrep, int64_t item, int phase,
                                              const uint32_t* __restrict__ perms, int& rep, int64_t& fid)
{
    int lo = 0, hi = nrep - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (descs[mid].items_off <= item) lo = mid; else hi = mid - 1;
    }
    const RepDesc& D = descs[lo];
    const int64_t local = item - D.items_off;
    const int colour = (int)((perms[lo] >> (4 * phase)) & 15u);
    int cnt[3], bit[3];
#pragma unroll
    for (int d = 0; d < 3; ++d) {
        bit[d] = (colour >> d) & 1;
        cnt[d] = D.nf[d] == 1 ? (bit[d] == 0 ? 1 : 0) : D.nf[d] / 2;
    }
    if (D.resident || local >= (int64_t)cnt[0] * cnt[1] * cnt[2]) return false;
    int fc[3];
    unflatten3(local, cnt[0], cnt[1], fc);
    const int f0 = D.nf[0] == 1 ? 0 : 2 * fc[0] + bit[0];
    const int f1 = D.nf[1] == 1 ? 0 : 2 * fc[1] + bit[1];
    const int f2 = D.nf[2] == 1 ? 0 : 2 * fc[2] + bit[2];
    rep = lo;
    fid = ((int64_t)f2 * D.nf[1] + f1) * D.nf[0] + f0;
    return true;
}

// Screen pass of a colour phase: one thread per fragment of the phase's colour
// (every replica).  Fragments with vacancies go to an active list together
// with their first Philox block, drawn here thirty-two fragments per warp
// instead of once per fragment-warp.  split = 1: fragments holding one or two
// vacancies go to lists of their own (act + total_items, act + 2 total_items;
// counters act_count[8 + phase], act_count[16 + phase]) for the grouped
// small-fragment pass; split = 2: cls[item] = 1 marks a fragment holding 1 to
// LANE_REG_MAX_V vacancies, left to the one-thread-per-fragment pass in
// registers; the rest (or all) go to act, act_count[phase].
template <int PREC>
__global__ void __launch_bounds__(256) k_screen(const RepDesc* __restrict__ descs, int nrep, int64_t total_items,
                                                int phase, unsigned long long* wctl,
                                                const uint32_t* __restrict__ perms,
                                                const int32_t* __restrict__ counts, ActEntry* act,
                                                int32_t* act_count, int split, uint8_t* cls)
{
    const int64_t item = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    // the window count advances here (nothing in this launch reads wctl[0])
    if (phase == 0 && item == 0) wctl[0] = wctl[1] + 1;
    bool keep = false;
    int list = 0;
    ActEntry e;
    int lo;
    int64_t fid;
    if (split == 2 && item < total_items) cls[item] = 0;
    if (item < total_items && item_fragment(descs, nrep, item, phase, perms, lo, fid)) {
        const RepDesc& D = descs[lo];
        const int nv = counts[D.frag_base + fid];
        const bool sparse = split == 2 && nv > 0 && nv <= LANE_REG_MAX_V;
        if (split == 2) cls[item] = sparse;
        if (nv > 0 && !sparse) {
            keep = true;
            list = split == 1 && nv <= 2 ? nv : 0;
            const uint64_t w = D.window + wctl[1];
            const U64x4 blk = philox4x64((uint64_t)fid, w, 0, 0, D.seed, key_word(D.replica, PURPOSE_HOP));
            e.rep = lo;
            e.nv = nv;
            e.fid = fid;
            e.xs[0] = blk.x[1];
            e.xs[1] = blk.x[3];
            if constexpr (PREC == 0) {
                e.E[0] = (uint64_t)__double_as_longlong(neglog64(blk.x[0]));
                e.E[1] = (uint64_t)__double_as_longlong(neglog64(blk.x[2]));
            } else {
                e.E[0] = (uint64_t)__float_as_uint(neglog32(blk.x[0]));
                e.E[1] = (uint64_t)__float_as_uint(neglog32(blk.x[2]));
            }
        }
    }
    // one atomic per warp and list for the slots of its kept fragments
    const int lane = threadIdx.x & 31;
    for (int l = 0; l < 3; ++l) {
        const bool mine = keep && list == l;
        const unsigned bal = __ballot_sync(0xffffffffu, mine);
        if (!bal) continue;
        int base = 0;
        if (lane == __ffs(bal) - 1) base = atomicAdd(act_count + 8 * l + phase, __popc(bal));
        base = __shfl_sync(0xffffffffu, base, __ffs(bal) - 1);
        if (mine) act[l * total_items + base + __popc(bal & ((1u << lane) - 1u))] = e;
    }
}

// Run pass of a colour phase: one warp per screened fragment (grid-stride):
// BKL on the fragment's vacancies until the next event would pass the window.
template <int PREC, bool SITE, bool GRAIN>
__global__ void __launch_bounds__(128, 8) k_run(const RepDesc* __restrict__ descs, const ActEntry* __restrict__ act,
                                             const int32_t* __restrict__ act_count, int phase,
                                             const unsigned long long* wctl, uint32_t* occ, VacRec* recs,
                                             int32_t* counts, int32_t* tracer, unsigned long long* stats,
                                             uint32_t* status, int cap, SiteArgs sa)
{
    static_assert(!SITE || PREC == 0, "site energies use the plain form");
    using A = Arith<PREC>;
    using V = typename A::V;
    extern __shared__ __align__(16) unsigned char smem[];
    const int lane = threadIdx.x & 31;
    const int wib = threadIdx.x >> 5;
    const int nact = act_count[phase];
    const int nwarps_grid = gridDim.x * (blockDim.x >> 5);
    for (int a = blockIdx.x * (blockDim.x >> 5) + wib; a < nact; a += nwarps_grid) {
    const ActEntry ent = act[a];
    const int lo = ent.rep;
    const RepDesc& D = descs[lo];
    const uint64_t w = D.window + wctl[1];
    const int64_t fid = ent.fid;
    int f[3], lo_c[3], hi_c[3];
    unflatten3(fid, D.nf[0], D.nf[1], f);
#pragma unroll
    for (int d = 0; d < 3; ++d) {
        lo_c[d] = frag_start(f[d], D.base[d], D.rem[d]);
        hi_c[d] = frag_start(f[d] + 1, D.base[d], D.rem[d]);
    }
    const int64_t g = D.frag_base + fid;

    int nv = ent.nv;  // the screen pass's count
    if (nv > cap) {
        if (lane == 0) atomicOr(status, STATUS_OVERFLOW);
        nv = cap;
    }
    WarpSmem S = carve(smem + warp_smem_bytes(cap, SITE) * wib, cap);

    // slots: the fragment's records in ascending site order
    for (int k = lane; k < nv; k += 32) S.rec[k] = recs[g * cap + k];
    __syncwarp();
    for (int k = lane; k < nv; k += 32) {
        const uint64_t mk = S.rec[k].key;
        int rank = 0;
        for (int o = 0; o < nv; ++o) rank += S.rec[o].key < mk;
        S.order[rank] = (uint16_t)k;
        S.alive[rank] = 1;
    }
    __syncwarp();
    const int nslots = nv;
    const int nch = (nslots + 3) >> 2;  // 32 events per chunk
    if constexpr (SITE) compute_rates_site<GRAIN>(D, occ, sa, S, nslots, nch, lane, status);
    else compute_types<GRAIN>(D, occ, S, nslots, nch, lane, sa.gbound);
    __syncwarp();
    // rate of event index e (lane-local chunk element)
    auto rate_of = [&](int e) -> V {
        if constexpr (SITE) return (V)S.rate[e];
        else return A::template rate<GRAIN>(D, S.types[e]);
    };

    const uint64_t hop_k1 = key_word(D.replica, PURPOSE_HOP);
    // draws for events [64*batch, 64*batch+64): lane l holds Philox block 32*batch + l
    uint64_t batch = ~0ull;
    uint64_t xs_even = 0, xs_odd = 0;
    double Ed_even = 0.0, Ed_odd = 0.0;
    float Ef_even = 0.f, Ef_odd = 0.f;

    double clock = 0.0;
    uint64_t i = 0;
    uint32_t nhand = 0;
    for (;;) {
        // totals: canonical scan over chunks with a running carry
        V carry = A::zero();
        V Plast = A::zero();
        for (int c = 0; c < nch; ++c) {
            const V v = rate_of(c * 32 + lane);
            const V p = A::add(carry, warp_scan<PREC>(v, lane));
            carry = A::shfl(p, 31);
            Plast = p;
        }
        const V total = carry;
        if (!A::pos(total)) break;
        if (i >= MAX_EVENTS_PER_PHASE) {
            if (lane == 0) atomicOr(status, STATUS_EVENT_LIMIT);
            break;
        }

        uint64_t xs;
        double Ed = 0.0;
        float Ef = 0.f;
        if (i < 2) {  // block 0, drawn by the screen pass
            xs = ent.xs[i];
            if constexpr (PREC == 0) Ed = __longlong_as_double((long long)ent.E[i]);
            else Ef = __uint_as_float((uint32_t)ent.E[i]);
        } else {
            // events [2 + 64 b, 66 + 64 b): blocks 1 + 32 b + lane
            const uint64_t k = i - 2;
            if ((k >> 6) != batch) {
                batch = k >> 6;
                const U64x4 blk = philox4x64((uint64_t)fid, w, 1 + 32 * batch + lane, 0, D.seed, hop_k1);
                xs_even = blk.x[1];
                xs_odd = blk.x[3];
                if constexpr (PREC == 0) {
                    Ed_even = neglog64(blk.x[0]);
                    Ed_odd = neglog64(blk.x[2]);
                } else {
                    Ef_even = neglog32(blk.x[0]);
                    Ef_odd = neglog32(blk.x[2]);
                }
            }
            const int src = (int)((k >> 1) & 31);
            const bool odd = (k & 1) != 0;
            xs = __shfl_sync(0xffffffffu, odd ? xs_odd : xs_even, src);
            if constexpr (PREC == 0) Ed = __shfl_sync(0xffffffffu, odd ? Ed_odd : Ed_even, src);
            else Ef = __shfl_sync(0xffffffffu, odd ? Ef_odd : Ef_even, src);
        }

        double dclock;
        int e_sel = -1;
        if constexpr (PREC == 0) {
            const double R = (double)total;
            const double dt = __ddiv_rn(Ed, R);
            if (__dadd_rn(clock, dt) > D.tau) break;
            dclock = dt;
            const double target = __dmul_rn(__dmul_rn(__ull2double_rn(xs >> 11), 0x1p-53), R);
            // first event with a nonzero rate whose prefix exceeds the target
            double cc = 0.0;
            for (int c = 0; c < nch; ++c) {
                double p;
                const double v = (double)rate_of(c * 32 + lane);
                if (nch == 1) {
                    p = (double)Plast;
                } else {
                    p = __dadd_rn(cc, warp_scan<0>(v, lane));
                    cc = __shfl_sync(0xffffffffu, p, 31);
                }
                const unsigned bal = __ballot_sync(0xffffffffu, v > 0.0 && p > target);
                if (bal) {
                    e_sel = c * 32 + __ffs(bal) - 1;
                    break;
                }
            }
            if (e_sel < 0) {  // rounding left no prefix above the target: last nonzero event
                for (int c = nch - 1; c >= 0 && e_sel < 0; --c) {
                    const unsigned bal = __ballot_sync(0xffffffffu, (double)rate_of(c * 32 + lane) > 0.0);
                    if (bal) e_sel = c * 32 + 31 - __clz(bal);
                }
            }
        } else {
            const unsigned long long Sq = (unsigned long long)total;
            const float ratio = __fdiv_rn(Ef, __ull2float_rn(Sq));
            const double dth = __dmul_rn((double)ratio, D.two_pow_F);
            if (__dadd_rn(clock, dth) > D.theta_tau) break;
            dclock = dth;
            const unsigned long long target = __umul64hi(xs, Sq);
            unsigned long long cc = 0ull;
            for (int c = 0; c < nch; ++c) {
                const unsigned long long v = (unsigned long long)rate_of(c * 32 + lane);
                unsigned long long p;
                if (nch == 1) {
                    p = (unsigned long long)Plast;
                } else {
                    p = cc + warp_scan<1>(v, lane);
                    cc = __shfl_sync(0xffffffffu, p, 31);
                }
                const unsigned bal = __ballot_sync(0xffffffffu, p > target);
                if (bal) {
                    e_sel = c * 32 + __ffs(bal) - 1;
                    break;
                }
            }
        }

        if constexpr (SITE) {
            // every lane moves part of the hopping vacancy's energy share
            int t, x, y, z;
            split_key(S.rec[S.order[e_sel >> 3]].key, t, x, y, z);
            const NbEntry nb = c_nb[t][e_sel & 7];
            move_field(D, sa, t, x, y, z, nb.t2, wrapc(x + nb.dc[0], D.L[0]), wrapc(y + nb.dc[1], D.L[1]),
                       wrapc(z + nb.dc[2], D.L[2]), lane);
            __syncwarp();  // every lane has read the record before lane 0 rewrites it
        }
        // apply the exchange (lane 0 writes; the rest of the warp waits)
        if (lane == 0) {
            const int m = e_sel >> 3, n = e_sel & 7;
            VacRec& r = S.rec[S.order[m]];
            int t, x, y, z;
            split_key(r.key, t, x, y, z);
            const NbEntry nb = c_nb[t][n];
            const int jx = wrapc(x + nb.dc[0], D.L[0]);
            const int jy = wrapc(y + nb.dc[1], D.L[1]);
            const int jz = wrapc(z + nb.dc[2], D.L[2]);
            const uint32_t ion = (uint32_t)((S.types[e_sel] % 6) / 3);
            atomicXor(occ + occ_word(D, t, x, y, z), ((uint32_t)SP_V ^ ion) << occ_shift(x));
            atomicXor(occ + occ_word(D, nb.t2, jx, jy, jz), (ion ^ (uint32_t)SP_V) << occ_shift(jx));
            r.d[0] += nb.d[0];
            r.d[1] += nb.d[1];
            r.d[2] += nb.d[2];
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
            r.key = make_key(nb.t2, jx, jy, jz);
            const bool owned = jx >= lo_c[0] && jx < hi_c[0] && jy >= lo_c[1] && jy < hi_c[1] &&
                               jz >= lo_c[2] && jz < hi_c[2];
            if (!owned) {
                const int gx = frag_of(jx, D.base[0], D.rem[0]);
                const int gy = frag_of(jy, D.base[1], D.rem[1]);
                const int gz = frag_of(jz, D.base[2], D.rem[2]);
                const int64_t g2 = D.frag_base + ((int64_t)gz * D.nf[1] + gy) * D.nf[0] + gx;
                const int slot = atomicAdd(counts + g2, 1);
                if (slot < cap) recs[g2 * cap + slot] = r;
                else atomicOr(status, STATUS_OVERFLOW);
                S.alive[m] = 0;
                ++nhand;
            }
            __threadfence_block();
        }
        if constexpr (SITE) __threadfence_block();  // field atomics before the rate reads
        __syncwarp();
        clock = __dadd_rn(clock, dclock);
        ++i;
        if constexpr (SITE) compute_rates_site<GRAIN>(D, occ, sa, S, nslots, nch, lane, status);
        else compute_types<GRAIN>(D, occ, S, nslots, nch, lane, sa.gbound);
        __syncwarp();
    }

    // surviving records stay with the fragment
    int base_pos = 0;
    for (int c = 0; c * 32 < nslots; ++c) {
        const int m = c * 32 + lane;
        const bool keep = m < nslots && S.alive[m];
        const unsigned bal = __ballot_sync(0xffffffffu, keep);
        if (keep) recs[g * cap + base_pos + __popc(bal & ((1u << lane) - 1u))] = S.rec[S.order[m]];
        base_pos += __popc(bal);
    }
    if (lane == 0) {
        counts[g] = base_pos;
        if (i) atomicAdd(stats + 2 * lo, (unsigned long long)i);
        if (nhand) atomicAdd(stats + 2 * lo + 1, (unsigned long long)nhand);
    }
    __syncwarp();  // the warp's shared memory is reused by its next fragment
    }
}

// Run pass for fragments holding one or two vacancies (table-rate path): a
// fragment takes a group of G = 8 nv lanes, lane = event index 8 slot +
// neighbour, and the groups of a warp (four of 8 lanes or two of 16) run in
// lock-step, so their memory round trips overlap and their instructions are
// issued once.  The group's Kogge-Stone scan over its G lanes yields the same
// partial sums as the general pass's 32-lane scan (strides of G and more only
// add the zero rates of empty lanes), the draws are the same Philox words
// (events 0, 1 from the screen pass, event i >= 2 from block 1 + (i-2)/2), and
// the selection and exchange are the same, so both passes compute the same
// trajectory.  Records and rate types live in registers.
template <int PREC, bool GRAIN>
__global__ void __launch_bounds__(128, 8) k_run_small(const RepDesc* __restrict__ descs,
                                                   const ActEntry* __restrict__ act, int64_t list_stride,
                                                   const int32_t* __restrict__ act_count, int phase,
                                                   const unsigned long long* wctl, uint32_t* occ, VacRec* recs,
                                                   int32_t* counts, int32_t* tracer, unsigned long long* stats,
                                                   uint32_t* status, int cap, const uint8_t* gb)
{
    using A = Arith<PREC>;
    using V = typename A::V;
    constexpr unsigned FULL = 0xffffffffu;
    const int lane = threadIdx.x & 31;
    const int n1 = act_count[8 + phase], n2 = act_count[16 + phase];
    const int items1 = (n1 + 3) >> 2;
    const int items = items1 + ((n2 + 1) >> 1);
    const int nwarps_grid = gridDim.x * (blockDim.x >> 5);
    for (int it = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5); it < items; it += nwarps_grid) {
        const bool two = it >= items1;  // warp-uniform: 2 x 16 lanes, else 4 x 8
        const int G = two ? 16 : 8;
        const int grp = two ? lane >> 4 : lane >> 3;
        const int sub = lane & (G - 1);
        const int n = sub & 7;
        const unsigned gmask = (two ? 0xffffu : 0xffu) << (grp * G);
        const int idx = two ? 2 * (it - items1) + grp : 4 * it + grp;
        const bool active = idx < (two ? n2 : n1);
        const ActEntry* list = act + (two ? 2 : 1) * list_stride;
        ActEntry ent{};
        if (active) ent = list[idx];
        const RepDesc& D = descs[ent.rep];
        const int64_t fid = ent.fid;
        const int64_t g = D.frag_base + fid;
        VacRec rec{};
        if (active) rec = recs[g * cap + (sub >> 3)];
        if (two) {  // slots in ascending site order: swap the halves' records if needed
            const uint64_t ok = __shfl_xor_sync(FULL, rec.key, 8);
            const int od0 = __shfl_xor_sync(FULL, rec.d[0], 8);
            const int od1 = __shfl_xor_sync(FULL, rec.d[1], 8);
            const int od2 = __shfl_xor_sync(FULL, rec.d[2], 8);
            const uint32_t oid = __shfl_xor_sync(FULL, rec.id, 8);
            const bool swap = (sub >> 3) == 0 ? ok < rec.key : rec.key < ok;
            if (swap) {
                rec.key = ok;
                rec.d[0] = od0;
                rec.d[1] = od1;
                rec.d[2] = od2;
                rec.id = oid;
            }
        }
        int lo_c[3] = {0, 0, 0}, hi_c[3] = {0, 0, 0};
        {
            int f[3];
            unflatten3(fid, D.nf[0], D.nf[1], f);
#pragma unroll
            for (int d = 0; d < 3; ++d) {
                lo_c[d] = frag_start(f[d], D.base[d], D.rem[d]);
                hi_c[d] = frag_start(f[d] + 1, D.base[d], D.rem[d]);
            }
        }
        const uint64_t w = D.window + wctl[1];
        bool alive = active;  // this lane's vacancy is still in the fragment
        int ty = -1;
        auto types = [&]() {
            ty = -1;
            if (alive) {
                int t, x, y, z;
                split_key(rec.key, t, x, y, z);
                const NbEntry nb = nb_entry(t, n);
                const int jx = wrapc(x + nb.dc[0], D.L[0]);
                const int jy = wrapc(y + nb.dc[1], D.L[1]);
                const int jz = wrapc(z + nb.dc[2], D.L[2]);
                const uint32_t word = __ldcg(occ + occ_word(D, nb.t2, jx, jy, jz));
                const int code = (int)((word >> occ_shift(jx)) & 3u);
                ty = code == SP_V ? -1 : code * 3 + nb.d[2] + 1;
                if constexpr (GRAIN) {
                    if (ty >= 0 && (gb[cell_index(D, x, y, z)] | gb[cell_index(D, jx, jy, jz)])) ty += 6;
                }
            }
        };
        types();
        double clock = 0.0;
        uint64_t i = 0;
        uint64_t xs_even = 0, xs_odd = 0;
        double Ed_even = 0.0, Ed_odd = 0.0;
        float Ef_even = 0.f, Ef_odd = 0.f;
        bool run = active;
        while (__any_sync(FULL, run)) {
            const V v = run ? A::template rate<GRAIN>(D, ty) : A::zero();
            V p = v;
#pragma unroll
            for (int off = 1; off < 16; off <<= 1) {
                if (off < G) {
                    const V t = __shfl_up_sync(FULL, p, off, G);
                    if (sub >= off) p = A::add(p, t);
                }
            }
            const V total = __shfl_sync(FULL, p, G - 1, G);
            bool go = run && A::pos(total);
            if (go && i >= MAX_EVENTS_PER_PHASE) {
                if (sub == 0) atomicOr(status, STATUS_EVENT_LIMIT);
                go = false;
            }
            uint64_t xs = 0;
            double Ed = 0.0;
            float Ef = 0.f;
            if (go) {
                if (i < 2) {
                    xs = ent.xs[i];
                    if constexpr (PREC == 0) Ed = __longlong_as_double((long long)ent.E[i]);
                    else Ef = __uint_as_float((uint32_t)ent.E[i]);
                } else {
                    const uint64_t k = i - 2;
                    if ((k & 1) == 0) {
                        const U64x4 blk = philox4x64((uint64_t)fid, w, 1 + (k >> 1), 0, D.seed,
                                                     key_word(D.replica, PURPOSE_HOP));
                        xs_even = blk.x[1];
                        xs_odd = blk.x[3];
                        if constexpr (PREC == 0) {
                            Ed_even = neglog64(blk.x[0]);
                            Ed_odd = neglog64(blk.x[2]);
                        } else {
                            Ef_even = neglog32(blk.x[0]);
                            Ef_odd = neglog32(blk.x[2]);
                        }
                    }
                    const bool odd = (k & 1) != 0;
                    xs = odd ? xs_odd : xs_even;
                    if constexpr (PREC == 0) Ed = odd ? Ed_odd : Ed_even;
                    else Ef = odd ? Ef_odd : Ef_even;
                }
            }
            double dclock = 0.0;
            bool cont;
            int e_sel;
            if constexpr (PREC == 0) {
                const double R = total;
                const double dt = go ? __ddiv_rn(Ed, R) : 0.0;
                cont = go && !(__dadd_rn(clock, dt) > D.tau);
                dclock = dt;
                const double target = __dmul_rn(__dmul_rn(__ull2double_rn(xs >> 11), 0x1p-53), R);
                const unsigned b1 = __ballot_sync(FULL, cont && v > 0.0 && p > target) & gmask;
                const unsigned b2 = __ballot_sync(FULL, cont && v > 0.0) & gmask;
                e_sel = b1 ? __ffs(b1) - 1 : (b2 ? 31 - __clz(b2) : -1);
            } else {
                const unsigned long long Sq = total;
                const float ratio = go ? __fdiv_rn(Ef, __ull2float_rn(Sq)) : 0.f;
                const double dth = __dmul_rn((double)ratio, D.two_pow_F);
                cont = go && !(__dadd_rn(clock, dth) > D.theta_tau);
                dclock = dth;
                const unsigned long long target = __umul64hi(xs, Sq);
                const unsigned b1 = __ballot_sync(FULL, cont && p > target) & gmask;
                e_sel = b1 ? __ffs(b1) - 1 : -1;
            }
            if (cont && lane == e_sel) {  // the selected event's own lane applies the exchange
                int t, x, y, z;
                split_key(rec.key, t, x, y, z);
                const NbEntry nb = nb_entry(t, n);
                const int jx = wrapc(x + nb.dc[0], D.L[0]);
                const int jy = wrapc(y + nb.dc[1], D.L[1]);
                const int jz = wrapc(z + nb.dc[2], D.L[2]);
                const uint32_t ion = (uint32_t)((ty % 6) / 3);
                atomicXor(occ + occ_word(D, t, x, y, z), ((uint32_t)SP_V ^ ion) << occ_shift(x));
                atomicXor(occ + occ_word(D, nb.t2, jx, jy, jz), (ion ^ (uint32_t)SP_V) << occ_shift(jx));
                rec.d[0] += nb.d[0];
                rec.d[1] += nb.d[1];
                rec.d[2] += nb.d[2];
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
                rec.key = make_key(nb.t2, jx, jy, jz);
                const bool owned = jx >= lo_c[0] && jx < hi_c[0] && jy >= lo_c[1] && jy < hi_c[1] &&
                                   jz >= lo_c[2] && jz < hi_c[2];
                if (!owned) {
                    const int gx = frag_of(jx, D.base[0], D.rem[0]);
                    const int gy = frag_of(jy, D.base[1], D.rem[1]);
                    const int gz = frag_of(jz, D.base[2], D.rem[2]);
                    const int64_t g2 = D.frag_base + ((int64_t)gz * D.nf[1] + gy) * D.nf[0] + gx;
                    const int slot = atomicAdd(counts + g2, 1);
                    if (slot < cap) recs[g2 * cap + slot] = rec;
                    else atomicOr(status, STATUS_OVERFLOW);
                    alive = false;
                }
                __threadfence_block();
            }
            __syncwarp();
            // the selected lane's record and flag go to the other lanes of its vacancy
            const int src = e_sel < 0 ? lane : e_sel;
            const uint64_t nkey = __shfl_sync(FULL, rec.key, src);
            const int nd0 = __shfl_sync(FULL, rec.d[0], src);
            const int nd1 = __shfl_sync(FULL, rec.d[1], src);
            const int nd2 = __shfl_sync(FULL, rec.d[2], src);
            const bool nalive = __shfl_sync(FULL, alive, src);
            if (cont && (src >> 3) == (lane >> 3)) {
                rec.key = nkey;
                rec.d[0] = nd0;
                rec.d[1] = nd1;
                rec.d[2] = nd2;
                alive = nalive;
            }
            if (cont) {
                clock = __dadd_rn(clock, dclock);
                ++i;
            }
            run = cont;
            if (run) types();
        }
        // surviving records stay with the fragment, in slot order
        const bool lead = active && n == 0;
        const unsigned surv = __ballot_sync(FULL, lead && alive) & gmask;
        if (lead && alive) recs[g * cap + __popc(surv & ((1u << lane) - 1u))] = rec;
        if (active && sub == 0) {
            const int kept = __popc(surv);
            counts[g] = kept;
            if (i) atomicAdd(stats + 2 * ent.rep, (unsigned long long)i);
            if (ent.nv > kept) atomicAdd(stats + 2 * ent.rep + 1, (unsigned long long)(ent.nv - kept));
        }
    }
}

// ------------------------------------------------------------------ one thread per fragment
// The neighbour table per site type for the one-thread-per-fragment pass:
// x, y = 8 bits per neighbour n (n-th byte): t2 | (dc_x+1) << 2 | (dc_y+1) << 4 |
// (dc_z+1) << 6; z = 2 bits per neighbour: d_z + 1.
__device__ __align__(16) uint4 g_lgeo[3];

// Rate types of the 8 events of the vacancy at `key` (mixed form), packed as
// nibbles n = type + 1 (0: no event), and the sum of their fixed-point rates.
// The 8 neighbour words are read from L2 (ld.global.cg: this thread's own
// exchanges are atomics there) before any is used.  Away from the lattice's
// faces no coordinate wraps, and a neighbour's row is the vacancy's row plus
// a 32-bit offset.
template <bool GRAIN>
__device__ __forceinline__ uint32_t lane_types(const RepDesc& D, const uint32_t* occ, const uint8_t* gb, uint64_t key,
                                               unsigned long long& sum)
{
    int t, x, y, z;
    split_key(key, t, x, y, z);
    const uint4 geo = __ldg(g_lgeo + t);
    const uint64_t g8 = ((uint64_t)geo.y << 32) | geo.x;
    const int L0 = D.L[0], L1 = D.L[1], L2 = D.L[2];
    const uint32_t* occ_r = occ + D.occ_word_off;
    const int64_t rw = D.row_words;
    uint32_t w[8];
    uint32_t xlo = 0;   // nibble n: x of neighbour n, mod 16
    uint32_t gbit = 0;  // grains: bit n set where neighbour n's cell is a boundary cell
    int64_t cells = 0;
    if constexpr (GRAIN) cells = D.site_off / 3;
    if (x >= 1 && x <= L0 - 2 && y >= 1 && y <= L1 - 2 && z >= 1 && z <= L2 - 2) {
        const int rb = z * L1 + y;
#pragma unroll
        for (int n = 0; n < 8; ++n) {
            const uint32_t f = (uint32_t)(g8 >> (8 * n));
            const int t2 = (int)(f & 3u);
            const int jx = x + (int)((f >> 2) & 3u) - 1;
            const int dcy = (int)((f >> 4) & 3u) - 1, dcz = (int)((f >> 6) & 3u) - 1;
            const int row = rb + dcz * L1 + dcy;
            w[n] = __ldcg(occ_r + ((int64_t)row * rw + (jx >> 4)) * 3 + t2);
            xlo |= (uint32_t)(jx & 15) << (4 * n);
            if constexpr (GRAIN)
                gbit |= (uint32_t)__ldg(gb + cells + ((int64_t)(z + dcz) * L1 + (y + dcy)) * L0 + jx) << n;
        }
    } else {
#pragma unroll
        for (int n = 0; n < 8; ++n) {
            const uint32_t f = (uint32_t)(g8 >> (8 * n));
            const int t2 = (int)(f & 3u);
            const int jx = wrapc(x + (int)((f >> 2) & 3u) - 1, L0);
            const int jy = wrapc(y + (int)((f >> 4) & 3u) - 1, L1);
            const int jz = wrapc(z + (int)((f >> 6) & 3u) - 1, L2);
            w[n] = __ldcg(occ_r + occ_index(rw, L1, t2, jx, jy, jz));
            xlo |= (uint32_t)(jx & 15) << (4 * n);
            if constexpr (GRAIN) gbit |= (uint32_t)__ldg(gb + cells + ((int64_t)jz * L1 + jy) * L0 + jx) << n;
        }
    }
    uint32_t gs = 0;
    if constexpr (GRAIN) gs = __ldg(gb + cells + ((int64_t)z * L1 + y) * L0 + x);
    uint32_t packed = 0;
    unsigned long long s = 0ull;
#pragma unroll
    for (int n = 0; n < 8; ++n) {
        const int code = (int)((w[n] >> (2 * ((xlo >> (4 * n)) & 15u))) & 3u);
        if (code != SP_V) {
            int ty = code * 3 + (int)((geo.z >> (2 * n)) & 3u);
            unsigned long long q;
            if constexpr (GRAIN) {
                if (gs | ((gbit >> n) & 1u)) {
                    q = D.qg[ty];
                    ty += 6;
                } else {
                    q = D.q[ty];
                }
            } else {
                q = D.q[ty];
            }
            s += q;
            packed |= (uint32_t)(ty + 1) << (4 * n);
        }
    }
    sum = s;
    return packed;
}

// Whether two O sites lie within one half-cell of each other along every axis
// (periodic): true for every pair of nearest neighbours.  A site's position in
// half-cells is 2 (x, y, z) + e_t.
__device__ __forceinline__ bool within_half_cell(const RepDesc& D, uint64_t a, uint64_t b)
{
    int ta, xa, ya, za, tb, xb, yb, zb;
    split_key(a, ta, xa, ya, za);
    split_key(b, tb, xb, yb, zb);
    const int h[3] = {2 * (xa - xb) + (ta == 0) - (tb == 0), 2 * (ya - yb) + (ta == 1) - (tb == 1),
                      2 * (za - zb) + (ta == 2) - (tb == 2)};
    bool near = true;
#pragma unroll
    for (int d = 0; d < 3; ++d) {
        int v = h[d];
        if (v > D.L[d]) v -= 2 * D.L[d];
        else if (v < -D.L[d]) v += 2 * D.L[d];
        near = near && v >= -1 && v <= 1;
    }
    return near;
}

__device__ __forceinline__ void order_pair(VacRec& a, VacRec& b)
{
    if (b.key < a.key) {
        const VacRec t = a;
        a = b;
        b = t;
    }
}

// One colour phase of the mixed form for the fragments the screen pass
// classed as sparse (one to LANE_REG_MAX_V vacancies): one thread per work
// item, with the fragment's records, packed rate types and per-vacancy rate
// sums in registers, so that a warp runs 32 fragments.  It runs beside the
// warp-per-fragment pass on the screen's list; the class byte (not the count,
// which that pass rewrites when it finishes a fragment) decides which pass
// owns a fragment.  The mixed form's sums are exact integers: the total and
// the first event whose inclusive prefix exceeds the target are those of the
// warp passes' scans over the same slot order (ascending site).  The draws
// are the same Philox words (event i: block i/2, words 1 and 0 for even i, 3
// and 2 for odd i), the window test, selection and exchange are the same, so
// the trajectory is the same.  After a hop only the moved vacancy and those
// within a half-cell of its old or new site re-read their neighbour words;
// every other rate is unchanged.
template <bool GRAIN>
__global__ void __launch_bounds__(128) k_run_lane_reg(const RepDesc* __restrict__ descs, int nrep,
                                                      int64_t total_items, int phase, const unsigned long long* wctl,
                                                      const uint32_t* __restrict__ perms,
                                                      const uint8_t* __restrict__ cls, uint32_t* occ, VacRec* recs,
                                                      int32_t* counts, int32_t* tracer, unsigned long long* stats,
                                                      uint32_t* status, int cap, const uint8_t* gb)
{
    constexpr int NL = LANE_REG_MAX_V;
    constexpr unsigned FULL = 0xffffffffu;
    const int64_t item = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    int rep = -1;
    int64_t fid = 0;
    int nv = 0;
    if (item < total_items && cls[item] && item_fragment(descs, nrep, item, phase, perms, rep, fid))
        nv = counts[descs[rep].frag_base + fid];
    uint32_t hops = 0, nhand = 0;
    if (nv > 0) {
        const RepDesc& D = descs[rep];
        const int64_t g = D.frag_base + fid;
        if (nv > cap) {
            atomicOr(status, STATUS_OVERFLOW);
            nv = cap;
        }
        // slots in ascending site order (a 4-input sorting network; empty slots last)
        VacRec r[NL];
#pragma unroll
        for (int k = 0; k < NL; ++k) {
            if (k < nv) {
                r[k] = recs[g * cap + k];
            } else {
                r[k].key = ~0ull;
                r[k].d[0] = r[k].d[1] = r[k].d[2] = 0;
                r[k].id = 0;
            }
        }
        static_assert(NL == 4, "sorting network for four slots");
        order_pair(r[0], r[1]);
        order_pair(r[2], r[3]);
        order_pair(r[0], r[2]);
        order_pair(r[1], r[3]);
        order_pair(r[1], r[2]);
        int lo_c[3], hi_c[3];
        {
            int f[3];
            unflatten3(fid, D.nf[0], D.nf[1], f);
#pragma unroll
            for (int d = 0; d < 3; ++d) {
                lo_c[d] = frag_start(f[d], D.base[d], D.rem[d]);
                hi_c[d] = frag_start(f[d] + 1, D.base[d], D.rem[d]);
            }
        }
        uint32_t ty[NL];
        unsigned long long sm[NL];
        uint32_t alive = (1u << nv) - 1u;
#pragma unroll
        for (int k = 0; k < NL; ++k) {
            sm[k] = 0ull;
            ty[k] = k < nv ? lane_types<GRAIN>(D, occ, gb, r[k].key, sm[k]) : 0u;
        }
        const uint64_t w = D.window + wctl[1];
        const uint64_t k1 = key_word(D.replica, PURPOSE_HOP);
        U64x4 blk{};
        double clock = 0.0;
        uint64_t i = 0;
        for (;;) {
            unsigned long long total = 0ull;
#pragma unroll
            for (int k = 0; k < NL; ++k) total += sm[k];
            if (total == 0ull) break;
            if (i >= MAX_EVENTS_PER_PHASE) {
                atomicOr(status, STATUS_EVENT_LIMIT);
                break;
            }
            if ((i & 1) == 0) blk = philox4x64((uint64_t)fid, w, i >> 1, 0, D.seed, k1);
            const bool odd = (i & 1) != 0;
            const uint64_t xs = odd ? blk.x[3] : blk.x[1];
            const float Ef = neglog32(odd ? blk.x[2] : blk.x[0]);
            const float ratio = __fdiv_rn(Ef, __ull2float_rn(total));
            const double dth = __dmul_rn((double)ratio, D.two_pow_F);
            if (__dadd_rn(clock, dth) > D.theta_tau) break;
            const unsigned long long target = __umul64hi(xs, total);
            // slot m and neighbour n of the first event whose prefix exceeds the target
            int m = NL - 1;
            unsigned long long acc = 0ull;
            bool found = false;
#pragma unroll
            for (int k = 0; k < NL; ++k) {
                if (!found) {
                    if (acc + sm[k] > target) {
                        m = k;
                        found = true;
                    } else {
                        acc += sm[k];
                    }
                }
            }
            VacRec cur = r[0];
            uint32_t tym = ty[0];
#pragma unroll
            for (int k = 1; k < NL; ++k) {
                if (k == m) {
                    cur = r[k];
                    tym = ty[k];
                }
            }
            int n = 7;
            found = false;
#pragma unroll
            for (int e = 0; e < 8; ++e) {
                const int nib = (int)((tym >> (4 * e)) & 15u);
                if (!found && nib) {
                    const int tv = nib - 1;
                    acc += GRAIN ? (tv < 6 ? D.q[tv] : D.qg[tv - 6]) : D.q[tv];
                    if (acc > target) {
                        n = e;
                        found = true;
                    }
                }
            }
            // the exchange
            const uint64_t s_key = cur.key;
            int t, x, y, z;
            split_key(s_key, t, x, y, z);
            const NbEntry nb = nb_entry(t, n);
            const int jx = wrapc(x + nb.dc[0], D.L[0]);
            const int jy = wrapc(y + nb.dc[1], D.L[1]);
            const int jz = wrapc(z + nb.dc[2], D.L[2]);
            const int tyv = (int)((tym >> (4 * n)) & 15u) - 1;
            const uint32_t ion = (uint32_t)((tyv % 6) / 3);
            atomicXor(occ + occ_word(D, t, x, y, z), ((uint32_t)SP_V ^ ion) << occ_shift(x));
            atomicXor(occ + occ_word(D, nb.t2, jx, jy, jz), (ion ^ (uint32_t)SP_V) << occ_shift(jx));
            cur.d[0] += nb.d[0];
            cur.d[1] += nb.d[1];
            cur.d[2] += nb.d[2];
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
            cur.key = make_key(nb.t2, jx, jy, jz);
            const bool owned = jx >= lo_c[0] && jx < hi_c[0] && jy >= lo_c[1] && jy < hi_c[1] && jz >= lo_c[2] &&
                               jz < hi_c[2];
            if (!owned) {
                const int gx = frag_of(jx, D.base[0], D.rem[0]);
                const int gy = frag_of(jy, D.base[1], D.rem[1]);
                const int gz = frag_of(jz, D.base[2], D.rem[2]);
                const int64_t g2 = D.frag_base + ((int64_t)gz * D.nf[1] + gy) * D.nf[0] + gx;
                const int slot = atomicAdd(counts + g2, 1);
                if (slot < cap) recs[g2 * cap + slot] = cur;
                else atomicOr(status, STATUS_OVERFLOW);
                alive &= ~(1u << m);
                ++nhand;
            }
            __threadfence_block();
#pragma unroll
            for (int k = 0; k < NL; ++k)
                if (k == m) r[k] = cur;
            clock = __dadd_rn(clock, dth);
            ++i;
            // rates after the exchange: vacancies near s or j read their words again
            uint32_t redo = 0;
#pragma unroll
            for (int k = 0; k < NL; ++k) {
                const bool live = (alive >> k) & 1u;
                if (!live) {
                    ty[k] = 0u;
                    sm[k] = 0ull;
                } else if (k == m || within_half_cell(D, r[k].key, s_key) || within_half_cell(D, r[k].key, cur.key)) {
                    redo |= 1u << k;
                }
            }
            while (redo) {
                const int k = __ffs(redo) - 1;
                redo &= redo - 1u;
                uint64_t kk = r[0].key;
#pragma unroll
                for (int q = 1; q < NL; ++q)
                    if (q == k) kk = r[q].key;
                unsigned long long sk = 0ull;
                const uint32_t tk = lane_types<GRAIN>(D, occ, gb, kk, sk);
#pragma unroll
                for (int q = 0; q < NL; ++q)
                    if (q == k) {
                        ty[q] = tk;
                        sm[q] = sk;
                    }
            }
        }
        hops = (uint32_t)i;
        // surviving records stay with the fragment, in slot order
        int pos = 0;
#pragma unroll
        for (int k = 0; k < NL; ++k)
            if ((alive >> k) & 1u) recs[g * cap + pos++] = r[k];
        counts[g] = pos;
    }
    // hop and hand-off counters: one atomic per warp where its fragments share a replica
    const int r0 = __shfl_sync(FULL, rep, 0);
    if (__all_sync(FULL, rep == r0 || (hops == 0 && nhand == 0)) && r0 >= 0) {
        const unsigned hs = __reduce_add_sync(FULL, hops), ns = __reduce_add_sync(FULL, nhand);
        if ((threadIdx.x & 31) == 0) {
            if (hs) atomicAdd(stats + 2 * r0, (unsigned long long)hs);
            if (ns) atomicAdd(stats + 2 * r0 + 1, (unsigned long long)ns);
        }
    } else {
        if (hops) atomicAdd(stats + 2 * rep, (unsigned long long)hops);
        if (nhand) atomicAdd(stats + 2 * rep + 1, (unsigned long long)nhand);
    }
}

// n-th (from 0) set bit of m; m holds more than n set bits
__device__ __forceinline__ int nth_set_bit(unsigned m, int n)
{
    int pos = 0;
#pragma unroll
    for (int w = 16; w >= 1; w >>= 1) {
        const int c = __popc((m >> pos) & ((1u << w) - 1u));
        if (n >= c) {
            n -= c;
            pos += w;
        }
    }
    return pos;
}

constexpr int LANE_THREADS = 128;

// The fragment slots of the lanes of one block in shared memory: slot k of
// thread x at [k][x], so that a warp's accesses to one slot are contiguous.
struct LaneSlots {
    unsigned long long key[LANE_MAX_V][LANE_THREADS];
    unsigned long long sum[LANE_MAX_V][LANE_THREADS];  // fixed-point rate sum of the slot's 8 events
    int32_t d[3][LANE_MAX_V][LANE_THREADS];
    uint32_t id[LANE_MAX_V][LANE_THREADS];
    uint32_t ty[LANE_MAX_V][LANE_THREADS];             // packed rate types (lane_types)
};

// asynchronous copies global -> shared (cp.async, 4 or 8 bytes, both addresses
// aligned to the size), completed for the issuing thread by cp_async_wait_all
__device__ __forceinline__ void cp_async4(void* smem, const void* gmem)
{
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4;" ::"r"((uint32_t)__cvta_generic_to_shared(smem)),
                 "l"(gmem)
                 : "memory");
}
__device__ __forceinline__ void cp_async8(void* smem, const void* gmem)
{
    asm volatile("cp.async.ca.shared.global [%0], [%1], 8;" ::"r"((uint32_t)__cvta_generic_to_shared(smem)),
                 "l"(gmem)
                 : "memory");
}
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_all;" ::: "memory"); }

__device__ __forceinline__ uint64_t shfl_u64(uint64_t v, int src)
{
    const unsigned lo = __shfl_sync(0xffffffffu, (unsigned)v, src);
    const unsigned hi = __shfl_sync(0xffffffffu, (unsigned)(v >> 32), src);
    return ((uint64_t)hi << 32) | lo;
}

// One colour phase of the mixed form for every fragment of the phase's colour,
// one fragment per lane at a time.  A persistent grid: the warps take windows
// of 32 consecutive work items (fragments) from a ticket counter, each
// window's vacancy counts loaded while the one before is in use and its
// ticket drawn a window earlier still.  Fragments holding
// more than LANE_MAX_V vacancies go to the warp-per-fragment pass (act list 0,
// with their first Philox block), which runs after this one.
//
// Each lane runs a small state machine, one step of each kind per loop turn:
//   take      a lane without a fragment takes the next one of the window that
//             holds 1..LANE_MAX_V vacancies: records to its shared-memory
//             slots, slot order = ascending site (a rank permutation), draw
//             block 0;
//   rates     one slot whose rate types are stale reads its 8 neighbour words;
//   event     the window test, then BKL selection and the exchange, or the
//             fragment's records are written back.
// A lane therefore moves on to its next fragment as soon as its current one
// ends, instead of waiting for the warp's longest event chain.
//
// Same trajectory as the warp passes: the mixed form's sums are exact
// integers, so the total and the first event whose inclusive prefix exceeds
// the target (slot order, then neighbour order) are those of their scans; the
// draws are the same Philox words (event i: block i/2, words 1 and 0 for even
// i, 3 and 2 for odd i); the window test, selection and exchange are the same.
// After a hop only the moved vacancy and those within a half-cell of its old
// or new site re-read their neighbour words; every other rate is unchanged.
template <bool GRAIN>
__global__ void __launch_bounds__(LANE_THREADS) k_run_lane(const RepDesc* __restrict__ descs, int nrep,
                                                           int64_t total_items, int phase, unsigned long long* wctl,
                                                           const uint32_t* __restrict__ perms, ActEntry* act,
                                                           int32_t* act_count, uint32_t* occ, VacRec* recs,
                                                           int32_t* counts, int32_t* tracer,
                                                           unsigned long long* stats, uint32_t* status, int cap,
                                                           const uint8_t* gb)
{
    constexpr int NL = LANE_MAX_V;
    static_assert(NL <= 8, "slot order packs 8 slot indices of 4 bits");
    constexpr unsigned FULL = 0xffffffffu;
    __shared__ LaneSlots S;
    const int tid = threadIdx.x, lane = tid & 31;
    const unsigned below = (1u << lane) - 1u;
    const uint64_t wk = wctl[1];
    // the window count advances here (nothing in this launch reads wctl[0])
    if (phase == 0 && blockIdx.x == 0 && tid == 0) wctl[0] = wk + 1;

    // windows of 32 items from the phase's ticket counter
    int32_t* ticket = act_count + 24 + phase;
    const int64_t nwin = (total_items + 31) / 32;
    auto item_count = [&](int64_t it, int& rp, int64_t& fd) -> int {
        if (it >= total_items || !item_fragment(descs, nrep, it, phase, perms, rp, fd)) return 0;
        return __ldcg(counts + descs[rp].frag_base + fd);
    };
    int64_t wbase = 0;   // window in use: lane l describes item wbase + l
    int64_t next_win;    // the next window (its counts are loading)
    int drawn = 0;       // lane 0: the ticket after it
    int cur_rep = 0, cur_cnt = 0;
    int64_t cur_fid = 0;
    unsigned avail = 0;  // window items not yet taken that hold 1..NL vacancies
    int next_cnt;
    {
        int t0 = 0;
        if (lane == 0) t0 = atomicAdd(ticket, 1);
        next_win = __shfl_sync(FULL, t0, 0);
        if (lane == 0) drawn = atomicAdd(ticket, 1);
        int rp;
        int64_t fd;
        next_cnt = item_count(next_win * 32 + lane, rp, fd);
    }

    // the lane's fragment
    bool active = false;
    int rep = 0, nv = 0;
    int64_t fid = 0, g = 0;
    uint64_t wnd = 0;
    uint32_t ord = 0, alive = 0, pending = 0, nhand = 0;
    int lo_c[3] = {0, 0, 0}, hi_c[3] = {0, 0, 0};
    U64x4 blk{};
    double clock = 0.0;
    uint64_t i = 0;
    // hop and hand-off counts of the lane, for replica acc_rep
    int acc_rep = -1;
    unsigned long long acc_hops = 0, acc_hand = 0;

    for (;;) {
        // ---- take: lanes without a fragment take the window's next ones
        for (;;) {
            const unsigned need = __ballot_sync(FULL, !active);
            if (need == 0) break;
            if (avail == 0) {
                if (next_win >= nwin) break;  // every window is taken
                wbase = next_win * 32;
                cur_cnt = next_cnt;
                if (!item_fragment(descs, nrep, wbase + lane, phase, perms, cur_rep, cur_fid)) cur_cnt = 0;
                next_win = __shfl_sync(FULL, drawn, 0);
                if (lane == 0 && next_win < nwin) drawn = atomicAdd(ticket, 1);
                {
                    int rp;
                    int64_t fd;
                    next_cnt = item_count(next_win * 32 + lane, rp, fd);
                }
                // fragments too dense for a lane: to the warp pass, with their first draws
                const bool big = cur_cnt > NL;
                const unsigned bal = __ballot_sync(FULL, big);
                if (bal) {
                    int base = 0;
                    if (lane == __ffs(bal) - 1) base = atomicAdd(act_count + phase, __popc(bal));
                    base = __shfl_sync(FULL, base, __ffs(bal) - 1);
                    if (big) {
                        const RepDesc& Dc = descs[cur_rep];
                        const U64x4 b0 = philox4x64((uint64_t)cur_fid, Dc.window + wk, 0, 0, Dc.seed,
                                                    key_word(Dc.replica, PURPOSE_HOP));
                        ActEntry e;
                        e.rep = cur_rep;
                        e.nv = cur_cnt;
                        e.fid = cur_fid;
                        e.xs[0] = b0.x[1];
                        e.xs[1] = b0.x[3];
                        e.E[0] = (uint64_t)__float_as_uint(neglog32(b0.x[0]));
                        e.E[1] = (uint64_t)__float_as_uint(neglog32(b0.x[2]));
                        act[base + __popc(bal & below)] = e;
                    }
                }
                avail = __ballot_sync(FULL, cur_cnt > 0 && cur_cnt <= NL);
                continue;
            }
            const int na = __popc(avail), take = min(na, __popc(need));
            const int k = __popc(need & below);
            const bool mine = !active && k < take;
            const int pos = mine ? nth_set_bit(avail, k) : lane;
            const int c = __shfl_sync(FULL, cur_cnt, pos);
            const int rp = __shfl_sync(FULL, cur_rep, pos);
            const uint64_t fd = shfl_u64((uint64_t)cur_fid, pos);
            avail = take == na ? 0u : avail & ~((2u << nth_set_bit(avail, take - 1)) - 1u);
            if (mine) {
                const RepDesc& D = descs[rp];
                rep = rp;
                fid = (int64_t)fd;
                g = D.frag_base + fid;
                nv = c;
                if (nv > cap) {
                    atomicOr(status, STATUS_OVERFLOW);
                    nv = cap;
                }
                // records to the slots, every copy in flight at once (one memory
                // latency instead of one per record); slot order by ascending site
                for (int q = 0; q < nv; ++q) {
                    const VacRec* src = recs + g * cap + q;
                    cp_async8(&S.key[q][tid], &src->key);
                    cp_async4(&S.d[0][q][tid], &src->d[0]);
                    cp_async4(&S.d[1][q][tid], &src->d[1]);
                    cp_async4(&S.d[2][q][tid], &src->d[2]);
                    cp_async4(&S.id[q][tid], &src->id);
                }
                cp_async_wait_all();
                uint32_t rank = 0;  // nibble k: rank of record k
                for (int q = 0; q < nv; ++q) {
                    const uint64_t kq = S.key[q][tid];
                    uint32_t rq = 0;
                    for (int j = 0; j < q; ++j) {
                        const bool less = S.key[j][tid] < kq;
                        rq += less;
                        rank += (uint32_t)(!less) << (4 * j);
                    }
                    rank |= rq << (4 * q);
                }
                ord = 0;
                for (int q = 0; q < nv; ++q) ord |= (uint32_t)q << (4 * ((rank >> (4 * q)) & 15u));
                int f[3];
                unflatten3(fid, D.nf[0], D.nf[1], f);
#pragma unroll
                for (int d = 0; d < 3; ++d) {
                    lo_c[d] = frag_start(f[d], D.base[d], D.rem[d]);
                    hi_c[d] = frag_start(f[d] + 1, D.base[d], D.rem[d]);
                }
                alive = pending = (1u << nv) - 1u;
                wnd = D.window + wk;
                blk = philox4x64((uint64_t)fid, wnd, 0, 0, D.seed, key_word(D.replica, PURPOSE_HOP));
                clock = 0.0;
                i = 0;
                nhand = 0;
                if (rep != acc_rep) {
                    if (acc_hops) atomicAdd(stats + 2 * acc_rep, acc_hops);
                    if (acc_hand) atomicAdd(stats + 2 * acc_rep + 1, acc_hand);
                    acc_hops = acc_hand = 0;
                    acc_rep = rep;
                }
                active = true;
            }
        }
        if (!__any_sync(FULL, active)) break;
        const RepDesc& D = descs[rep];

        // ---- rates: one stale slot
        if (active && pending) {
            const int k = __ffs(pending) - 1;
            pending &= pending - 1u;
            unsigned long long sk;
            S.ty[k][tid] = lane_types<GRAIN>(D, occ, gb, S.key[k][tid], sk);
            S.sum[k][tid] = sk;
        }

        // ---- event: the window test, then selection and exchange, or the end of the visit
        if (active && !pending) {
            unsigned long long total = 0ull;
            for (int k = 0; k < nv; ++k)
                if ((alive >> k) & 1u) total += S.sum[k][tid];
            bool fin = total == 0ull;
            if (!fin && i >= MAX_EVENTS_PER_PHASE) {
                atomicOr(status, STATUS_EVENT_LIMIT);
                fin = true;
            }
            if (!fin) {
                if ((i & 1) == 0 && i > 0)
                    blk = philox4x64((uint64_t)fid, wnd, i >> 1, 0, D.seed, key_word(D.replica, PURPOSE_HOP));
                const bool odd = (i & 1) != 0;
                const uint64_t xs = odd ? blk.x[3] : blk.x[1];
                const float Ef = neglog32(odd ? blk.x[2] : blk.x[0]);
                const float ratio = __fdiv_rn(Ef, __ull2float_rn(total));
                const double dth = __dmul_rn((double)ratio, D.two_pow_F);
                if (__dadd_rn(clock, dth) > D.theta_tau) {
                    fin = true;
                } else {
                    // slot m and neighbour n of the first event whose prefix exceeds the target
                    const unsigned long long target = __umul64hi(xs, total);
                    unsigned long long acc = 0ull;
                    int m = (int)(ord & 15u);
                    for (int sl = 0; sl < nv; ++sl) {
                        const int k = (int)((ord >> (4 * sl)) & 15u);
                        if ((alive >> k) & 1u) {
                            const unsigned long long sk = S.sum[k][tid];
                            m = k;
                            if (acc + sk > target) break;
                            acc += sk;
                        }
                    }
                    const uint32_t tym = S.ty[m][tid];
                    int n = 7;
#pragma unroll
                    for (int e = 0; e < 8; ++e) {
                        const int nib = (int)((tym >> (4 * e)) & 15u);
                        if (nib) {
                            const int tv = nib - 1;
                            acc += GRAIN ? (tv < 6 ? D.q[tv] : D.qg[tv - 6]) : D.q[tv];
                            if (acc > target) {
                                n = e;
                                break;
                            }
                        }
                    }
                    // the exchange
                    const uint64_t s_key = S.key[m][tid];
                    int t, x, y, z;
                    split_key(s_key, t, x, y, z);
                    const NbEntry nb = nb_entry(t, n);
                    const int jx = wrapc(x + nb.dc[0], D.L[0]);
                    const int jy = wrapc(y + nb.dc[1], D.L[1]);
                    const int jz = wrapc(z + nb.dc[2], D.L[2]);
                    const int tyv = (int)((tym >> (4 * n)) & 15u) - 1;
                    const uint32_t ion = (uint32_t)((tyv % 6) / 3);
                    atomicXor(occ + occ_word(D, t, x, y, z), ((uint32_t)SP_V ^ ion) << occ_shift(x));
                    atomicXor(occ + occ_word(D, nb.t2, jx, jy, jz), (ion ^ (uint32_t)SP_V) << occ_shift(jx));
                    const int d0 = S.d[0][m][tid] + nb.d[0];
                    const int d1 = S.d[1][m][tid] + nb.d[1];
                    const int d2 = S.d[2][m][tid] + nb.d[2];
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
                    const uint64_t j_key = make_key(nb.t2, jx, jy, jz);
                    const bool owned = jx >= lo_c[0] && jx < hi_c[0] && jy >= lo_c[1] && jy < hi_c[1] &&
                                       jz >= lo_c[2] && jz < hi_c[2];
                    if (owned) {
                        S.key[m][tid] = j_key;
                        S.d[0][m][tid] = d0;
                        S.d[1][m][tid] = d1;
                        S.d[2][m][tid] = d2;
                    } else {
                        const int gx = frag_of(jx, D.base[0], D.rem[0]);
                        const int gy = frag_of(jy, D.base[1], D.rem[1]);
                        const int gz = frag_of(jz, D.base[2], D.rem[2]);
                        const int64_t g2 = D.frag_base + ((int64_t)gz * D.nf[1] + gy) * D.nf[0] + gx;
                        const int slot = atomicAdd(counts + g2, 1);
                        if (slot < cap) {
                            VacRec r;
                            r.key = j_key;
                            r.d[0] = d0;
                            r.d[1] = d1;
                            r.d[2] = d2;
                            r.id = S.id[m][tid];
                            recs[g2 * cap + slot] = r;
                        } else {
                            atomicOr(status, STATUS_OVERFLOW);
                        }
                        alive &= ~(1u << m);
                        ++nhand;
                    }
                    __threadfence_block();
                    clock = __dadd_rn(clock, dth);
                    ++i;
                    // stale rates: the moved vacancy's, and those of vacancies near s or j
                    pending = owned ? 1u << m : 0u;
                    for (int k = 0; k < nv; ++k) {
                        if (k != m && ((alive >> k) & 1u)) {
                            const uint64_t kk = S.key[k][tid];
                            if (within_half_cell(D, kk, s_key) || within_half_cell(D, kk, j_key)) pending |= 1u << k;
                        }
                    }
                }
            }
            if (fin) {
                // surviving records stay with the fragment, in slot order
                int pos = 0;
                for (int sl = 0; sl < nv; ++sl) {
                    const int k = (int)((ord >> (4 * sl)) & 15u);
                    if ((alive >> k) & 1u) {
                        VacRec r;
                        r.key = S.key[k][tid];
                        r.d[0] = S.d[0][k][tid];
                        r.d[1] = S.d[1][k][tid];
                        r.d[2] = S.d[2][k][tid];
                        r.id = S.id[k][tid];
                        recs[g * cap + pos++] = r;
                    }
                }
                counts[g] = pos;
                acc_hops += i;
                acc_hand += nhand;
                active = false;
            }
        }
    }
    // counters: one atomic per warp where its lanes share a replica
    const int r0 = __shfl_sync(FULL, acc_rep, 0);
    if (__all_sync(FULL, acc_rep == r0 || (acc_hops == 0 && acc_hand == 0)) && r0 >= 0) {
        unsigned long long hs = acc_hops, ns = acc_hand;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            hs += __shfl_xor_sync(FULL, hs, o);
            ns += __shfl_xor_sync(FULL, ns, o);
        }
        if (lane == 0) {
            if (hs) atomicAdd(stats + 2 * r0, hs);
            if (ns) atomicAdd(stats + 2 * r0 + 1, ns);
        }
    } else {
        if (acc_hops) atomicAdd(stats + 2 * acc_rep, acc_hops);
        if (acc_hand) atomicAdd(stats + 2 * acc_rep + 1, acc_hand);
    }
}

// ------------------------------------------------------------------ site energies
// Dopant placement: cells f(0..n_fe-1) of a keyed Feistel bijection of the
// cell indices (the vacancy placement's construction, its own key).
__global__ void k_init_dopants(RepDesc D, int b_bits, int64_t n_fe, uint8_t* fe)
{
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n_fe) return;
    const uint64_t ncell = (uint64_t)D.L[0] * D.L[1] * D.L[2];
    const uint64_t mask = (1ull << b_bits) - 1ull;
    const uint64_t k0 = D.seed, k1 = key_word(D.replica, PURPOSE_DOPE);
    uint64_t v = (uint64_t)i;
    do {
        uint64_t Lh = v >> b_bits, Rh = v & mask;
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            const U64x4 o = philox4x64(Rh, (uint64_t)k, 0, 0, k0, k1);
            const uint64_t nr = Lh ^ (o.x[0] & mask);
            Lh = Rh;
            Rh = nr;
        }
        v = (Lh << b_bits) | Rh;
    } while (v >= ncell);
    fe[D.site_off / 3 + (int64_t)v] = 1;
}

__device__ __forceinline__ int replica_of(const RepDesc* descs, int nrep, int64_t v, bool by_cell)
{
    int lo = 0, hi = nrep - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        const int64_t start = by_cell ? descs[mid].site_off / 3 : descs[mid].frag_base;
        if (start <= v) lo = mid; else hi = mid - 1;
    }
    return lo;
}

// Energy field from the vacancies: each record adds its shell energies to the
// O sites around it (the field starts at zero).
__global__ void k_field_vac(const RepDesc* __restrict__ descs, int nrep, const VacRec* recs,
                            const int32_t* counts, int64_t nfrag_total, int cap, SiteArgs sa)
{
    const int64_t total = nfrag_total * cap;
    for (int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; k < total;
         k += (int64_t)gridDim.x * blockDim.x) {
        const int64_t g = k / cap;
        const int slot = (int)(k % cap);
        if (slot >= counts[g]) continue;
        const RepDesc& D = descs[replica_of(descs, nrep, g, false)];
        int t, x, y, z;
        split_key(recs[g * cap + slot].key, t, x, y, z);
        int32_t* field = sa.field + D.site_off;
        for (int o = 0; o < sa.n_vv; ++o) {
            const SiteOff a = sa.vv[t * SITE_MAX_VV + o];
            atomicAdd(field + site_lin(D, a.t2, wrapc(x + a.dc[0], D.L[0]), wrapc(y + a.dc[1], D.L[1]),
                                       wrapc(z + a.dc[2], D.L[2])),
                      a.e);
        }
    }
}

// Energy field from the dopants: each doped B site adds its shell energies to
// the O sites around it.
__global__ void k_field_dopant(const RepDesc* __restrict__ descs, int nrep, const uint8_t* fe, int64_t ncell_total,
                               const SiteOff* bo, int n_bo, int32_t* field_all)
{
    for (int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; c < ncell_total;
         c += (int64_t)gridDim.x * blockDim.x) {
        if (!fe[c]) continue;
        const RepDesc& D = descs[replica_of(descs, nrep, c, true)];
        const int64_t local = c - D.site_off / 3;
        const int x = (int)(local % D.L[0]);
        const int y = (int)((local / D.L[0]) % D.L[1]);
        const int z = (int)(local / ((int64_t)D.L[0] * D.L[1]));
        int32_t* field = field_all + D.site_off;
        for (int o = 0; o < n_bo; ++o) {
            const SiteOff a = bo[o];
            atomicAdd(field + site_lin(D, a.t2, wrapc(x + a.dc[0], D.L[0]), wrapc(y + a.dc[1], D.L[1]),
                                       wrapc(z + a.dc[2], D.L[2])),
                      a.e);
        }
    }
}

// ------------------------------------------------------------------ grains
// Seed g of a replica's Voronoi tessellation at X_d = mulhi(y_d, 256 L_d)
// (1/256-cell units), y = Philox block (g, 0, 0, 0) of (seed, replica, GRAIN).
__global__ void k_grain_seeds(const RepDesc* __restrict__ descs, int nrep, int n_grains, int64_t* X)
{
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= (int64_t)nrep * n_grains) return;
    const int r = (int)(i / n_grains), g = (int)(i % n_grains);
    const RepDesc& D = descs[r];
    const U64x4 y = philox4x64((uint64_t)g, 0, 0, 0, D.seed, key_word(D.replica, PURPOSE_GRAIN));
#pragma unroll
    for (int d = 0; d < 3; ++d) X[3 * i + d] = (int64_t)__umul64hi(y.x[d], 256ull * (uint64_t)D.L[d]);
}

// Grain of every cell: the nearest seed by squared minimum-image distance from
// the cell centre 256 c + 128 (exact integers; ties to the smaller seed).
__global__ void k_grain_map(const RepDesc* __restrict__ descs, int nrep, int64_t ncell_total, int n_grains,
                            const int64_t* __restrict__ X, int32_t* grain)
{
    for (int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; c < ncell_total;
         c += (int64_t)gridDim.x * blockDim.x) {
        int lo = 0, hi = nrep - 1;
        while (lo < hi) {
            const int mid = (lo + hi + 1) >> 1;
            if (descs[mid].site_off / 3 <= c) lo = mid; else hi = mid - 1;
        }
        const RepDesc& D = descs[lo];
        const int64_t local = c - D.site_off / 3;
        const int64_t cc[3] = {local % D.L[0], (local / D.L[0]) % D.L[1], local / ((int64_t)D.L[0] * D.L[1])};
        const int64_t* Xr = X + 3 * (int64_t)lo * n_grains;
        int best = 0;
        int64_t bd = INT64_MAX;
        for (int g = 0; g < n_grains; ++g) {
            int64_t d2 = 0;
#pragma unroll
            for (int d = 0; d < 3; ++d) {
                const int64_t box = 256 * (int64_t)D.L[d];
                int64_t dd = 256 * cc[d] + 128 - Xr[3 * g + d];
                dd = dd < 0 ? -dd : dd;
                dd = box - dd < dd ? box - dd : dd;
                d2 += dd * dd;
            }
            if (d2 < bd) {
                bd = d2;
                best = g;
            }
        }
        grain[c] = best;
    }
}

// Boundary layer: a cell with a cell of another grain within Chebyshev distance w.
__global__ void k_grain_boundary(const RepDesc* __restrict__ descs, int nrep, int64_t ncell_total, int w,
                                 const int32_t* __restrict__ grain, uint8_t* gb)
{
    for (int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; c < ncell_total;
         c += (int64_t)gridDim.x * blockDim.x) {
        int lo = 0, hi = nrep - 1;
        while (lo < hi) {
            const int mid = (lo + hi + 1) >> 1;
            if (descs[mid].site_off / 3 <= c) lo = mid; else hi = mid - 1;
        }
        const RepDesc& D = descs[lo];
        const int64_t c0 = D.site_off / 3, local = c - c0;
        const int x = (int)(local % D.L[0]), y = (int)((local / D.L[0]) % D.L[1]);
        const int z = (int)(local / ((int64_t)D.L[0] * D.L[1]));
        const int32_t own = grain[c];
        uint8_t b = 0;
        for (int dz = -w; dz <= w && !b; ++dz)
            for (int dy = -w; dy <= w && !b; ++dy)
                for (int dx = -w; dx <= w && !b; ++dx)
                    b = grain[c0 + ((int64_t)wrapc(z + dz, D.L[2]) * D.L[1] + wrapc(y + dy, D.L[1])) * D.L[0] +
                              wrapc(x + dx, D.L[0])] != own;
        gb[c] = b;
    }
}

cudaError_t launch_grains(const RepDesc* d_descs, int nrep, int64_t ncell_total, int n_grains, int width, int64_t* X,
                          int32_t* grain, uint8_t* gb, cudaStream_t st)
{
    const int threads = 256;
    const int64_t ns = (int64_t)nrep * n_grains;
    k_grain_seeds<<<(unsigned)((ns + threads - 1) / threads), threads, 0, st>>>(d_descs, nrep, n_grains, X);
    const unsigned blocks = (unsigned)std::min<int64_t>(65536, (ncell_total + threads - 1) / threads);
    k_grain_map<<<blocks, threads, 0, st>>>(d_descs, nrep, ncell_total, n_grains, X, grain);
    k_grain_boundary<<<blocks, threads, 0, st>>>(d_descs, nrep, ncell_total, width, grain, gb);
    return cudaGetLastError();
}

// ------------------------------------------------------------------ moments
// Vacancy records: out += {count, sum d, sum d^2} (two's-complement u64 atomics).
__global__ void k_moments_vac(const VacRec* recs, const int32_t* counts, int64_t frag0, int64_t nfrag,
                              int cap, unsigned long long* out)
{
    __shared__ unsigned long long acc[7];
    if (threadIdx.x < 7) acc[threadIdx.x] = 0ull;
    __syncthreads();
    unsigned long long a[7] = {0, 0, 0, 0, 0, 0, 0};
    const int64_t total = nfrag * cap;
    for (int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; k < total;
         k += (int64_t)gridDim.x * blockDim.x) {
        const int64_t f = k / cap;
        const int s = (int)(k % cap);
        if (s < counts[frag0 + f]) {
            const VacRec r = recs[(frag0 + f) * cap + s];
            a[0] += 1ull;
#pragma unroll
            for (int d = 0; d < 3; ++d) {
                a[1 + d] += (unsigned long long)(long long)r.d[d];
                a[4 + d] += (unsigned long long)((long long)r.d[d] * r.d[d]);
            }
        }
    }
#pragma unroll
    for (int q = 0; q < 7; ++q) {
        unsigned long long v = a[q];
        for (int off = 16; off; off >>= 1) v += __shfl_down_sync(0xffffffffu, v, off);
        if ((threadIdx.x & 31) == 0 && v) atomicAdd(acc + q, v);
    }
    __syncthreads();
    if (threadIdx.x < 7 && acc[threadIdx.x]) atomicAdd(out + threadIdx.x, acc[threadIdx.x]);
}

// Vacancy moments of every replica of the batch in one launch: blockIdx.y is
// the replica, blockIdx.x a chunk of its record slots; each block reduces in
// registers and shared memory and adds its 7 sums to out[7 r + q] once.
constexpr int MOM_THREADS = 256;
constexpr int MOM_SLOTS_PER_THREAD = 16;

__global__ void __launch_bounds__(MOM_THREADS) k_moments_vac_all(const RepDesc* __restrict__ descs,
                                                                 const VacRec* recs, const int32_t* counts,
                                                                 int cap, unsigned long long* out)
{
    __shared__ unsigned long long acc[7];
    const int r = blockIdx.y;
    const RepDesc& D = descs[r];
    const int64_t nfrag = (int64_t)D.nf[0] * D.nf[1] * D.nf[2];
    const int64_t total = nfrag * cap;
    const int64_t begin = (int64_t)blockIdx.x * MOM_THREADS * MOM_SLOTS_PER_THREAD;
    if (begin >= total) return;  // block-uniform
    if (threadIdx.x < 7) acc[threadIdx.x] = 0ull;
    __syncthreads();
    unsigned long long a[7] = {0, 0, 0, 0, 0, 0, 0};
    const int64_t end = min(total, begin + (int64_t)MOM_THREADS * MOM_SLOTS_PER_THREAD);
    for (int64_t k = begin + threadIdx.x; k < end; k += MOM_THREADS) {
        const int64_t f = D.frag_base + k / cap;
        const int s = (int)(k % cap);
        if (s >= counts[f]) continue;
        const VacRec v = recs[f * cap + s];
        a[0] += 1ull;
#pragma unroll
        for (int d = 0; d < 3; ++d) {
            a[1 + d] += (unsigned long long)(long long)v.d[d];
            a[4 + d] += (unsigned long long)((long long)v.d[d] * v.d[d]);
        }
    }
#pragma unroll
    for (int q = 0; q < 7; ++q) {
        unsigned long long v = a[q];
        for (int off = 16; off; off >>= 1) v += __shfl_down_sync(0xffffffffu, v, off);
        if ((threadIdx.x & 31) == 0 && v) atomicAdd(acc + q, v);
    }
    __syncthreads();
    if (threadIdx.x < 7 && acc[threadIdx.x]) atomicAdd(out + 7 * (int64_t)r + threadIdx.x, acc[threadIdx.x]);
}

// Tracer field over the sites holding `species`.
__global__ void k_moments_ion(RepDesc D, const uint32_t* occ, const int32_t* tracer, int species,
                              unsigned long long* out)
{
    __shared__ unsigned long long acc[7];
    if (threadIdx.x < 7) acc[threadIdx.x] = 0ull;
    __syncthreads();
    unsigned long long a[7] = {0, 0, 0, 0, 0, 0, 0};
    for (int64_t s = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; s < D.nsite;
         s += (int64_t)gridDim.x * blockDim.x) {
        const int x = (int)(s % D.L[0]);
        const int64_t rest = s / D.L[0];
        const int y = (int)(rest % D.L[1]);
        const int z = (int)((rest / D.L[1]) % D.L[2]);
        const int t = (int)(rest / ((int64_t)D.L[1] * D.L[2]));
        const uint32_t wv = occ[occ_word(D, t, x, y, z)];
        if ((int)((wv >> occ_shift(x)) & 3u) != species) continue;
        const int32_t* d = tracer + 3 * (D.site_off + s);
        a[0] += 1ull;
#pragma unroll
        for (int k = 0; k < 3; ++k) {
            a[1 + k] += (unsigned long long)(long long)d[k];
            a[4 + k] += (unsigned long long)((long long)d[k] * d[k]);
        }
    }
#pragma unroll
    for (int q = 0; q < 7; ++q) {
        unsigned long long v = a[q];
        for (int off = 16; off; off >>= 1) v += __shfl_down_sync(0xffffffffu, v, off);
        if ((threadIdx.x & 31) == 0 && v) atomicAdd(acc + q, v);
    }
    __syncthreads();
    if (threadIdx.x < 7 && acc[threadIdx.x]) atomicAdd(out + threadIdx.x, acc[threadIdx.x]);
}

// ------------------------------------------------------------------ launchers
cudaError_t upload_neighbours(const NbEntry* host)
{
    uint4 lg[3];
    for (int t = 0; t < 3; ++t) {
        uint64_t g8 = 0;
        uint32_t dz = 0;
        for (int n = 0; n < 8; ++n) {
            const NbEntry& e = host[8 * t + n];
            const uint64_t f = (uint64_t)e.t2 | (uint64_t)(e.dc[0] + 1) << 2 | (uint64_t)(e.dc[1] + 1) << 4 |
                               (uint64_t)(e.dc[2] + 1) << 6;
            g8 |= f << (8 * n);
            dz |= (uint32_t)(e.d[2] + 1) << (2 * n);
        }
        lg[t] = make_uint4((uint32_t)g8, (uint32_t)(g8 >> 32), dz, 0u);
    }
    cudaError_t e = cudaMemcpyToSymbol(c_nb, host, sizeof(NbEntry) * 24);
    if (e == cudaSuccess) e = cudaMemcpyToSymbol(g_nb, host, sizeof(NbEntry) * 24);
    return e != cudaSuccess ? e : cudaMemcpyToSymbol(g_lgeo, lg, sizeof lg);
}

cudaError_t launch_init(const RepDesc& D, int b_bits, int64_t n_vac, int64_t n_total, uint32_t* occ,
                        VacRec* recs, int32_t* counts, int cap, uint32_t* status, cudaStream_t st)
{
    if (n_total <= 0) return cudaSuccess;
    const int threads = 256;
    const int64_t blocks = (n_total + threads - 1) / threads;
    k_init<<<(unsigned)blocks, threads, 0, st>>>(D, b_bits, n_vac, n_total, occ, recs, counts, cap,
                                                 status);
    return cudaGetLastError();
}

size_t phase_smem_bytes(int cap, bool site) { return warp_smem_bytes(cap, site) * 4; }

using RunFn = void (*)(const RepDesc*, const ActEntry*, const int32_t*, int, const unsigned long long*, uint32_t*,
                      VacRec*, int32_t*, int32_t*, unsigned long long*, uint32_t*, int, SiteArgs);

// the run-pass instantiation for an arithmetic form, the site-energy path and grains
static RunFn run_kernel(int prec, bool site, bool grain)
{
    if (site) return grain ? k_run<0, true, true> : k_run<0, true, false>;
    if (prec == 0) return grain ? k_run<0, false, true> : k_run<0, false, false>;
    return grain ? k_run<1, false, true> : k_run<1, false, false>;
}

// The small-fragment pass runs beside the general one where a phase holds
// enough fragments to fill both: on a 1000^3 lattice (244k fragments per phase)
// it gains 15%, on 128^3 (512 per phase) the two extra launches per phase cost
// 20% (A/B on one GB300, identical hop counts).  It has no site energies.
bool window_split(bool site, int64_t total_items, int mode)
{
    return !site && (mode > 0 || (mode == 0 && total_items >= SPLIT_MIN_ITEMS));
}

// The mixed form runs its small fragments one thread per fragment, unless the
// grouped pass is asked for (small_pass 2): in registers beside the general
// pass, or, on phases of LANE_PERSIST_ITEMS fragments or more, in the
// persistent form (up to LANE_MAX_V vacancies in shared memory, the general
// pass after it).  On the bias cube (0.1% V, edge 8, n_tau 0.5; A/B on one
// GB300, identical hop counts) the register form ran 1.07e9 / 1.15e9 /
// 1.19e9 / 1.23e9 hops/s on 1000^3 / 1400^3 / 1800^3 / 2500^3, the
// persistent form 0.86e9 / 1.18e9 / 1.32e9 / 1.42e9.
int window_lane(int prec, int mode, int form, int64_t total_items)
{
    if (prec != 1 || mode == 2) return LANE_NONE;
    if (form == 1) return LANE_REGISTERS;
    if (form == 2) return LANE_PERSISTENT;
    return total_items >= LANE_PERSIST_ITEMS ? LANE_PERSISTENT : LANE_REGISTERS;
}

using LaneFn = void (*)(const RepDesc*, int, int64_t, int, unsigned long long*, const uint32_t*, ActEntry*, int32_t*,
                        uint32_t*, VacRec*, int32_t*, int32_t*, unsigned long long*, uint32_t*, int, const uint8_t*);
using LaneRegFn = void (*)(const RepDesc*, int, int64_t, int, const unsigned long long*, const uint32_t*,
                           const uint8_t*, uint32_t*, VacRec*, int32_t*, int32_t*, unsigned long long*, uint32_t*, int,
                           const uint8_t*);

static LaneFn lane_kernel(bool grain) { return grain ? k_run_lane<true> : k_run_lane<false>; }

using SmallFn = void (*)(const RepDesc*, const ActEntry*, int64_t, const int32_t*, int, const unsigned long long*,
                        uint32_t*, VacRec*, int32_t*, int32_t*, unsigned long long*, uint32_t*, int, const uint8_t*);

static SmallFn small_kernel(int prec, bool grain)
{
    if (prec == 0) return grain ? k_run_small<0, true> : k_run_small<0, false>;
    return grain ? k_run_small<1, true> : k_run_small<1, false>;
}

cudaError_t phase_prepare(int cap)
{
    cudaError_t e = cudaSuccess;
    for (int prec = 0; prec < 2; ++prec)
        for (int site = 0; site < 2; ++site)
            for (int grain = 0; grain < 2; ++grain) {
                if (site && prec) continue;
                if (e == cudaSuccess)
                    e = cudaFuncSetAttribute(run_kernel(prec, site, grain), cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             (int)phase_smem_bytes(cap, site));
            }
    return e;
}

// Blocks of the run pass: as many as fit on the GPU at once (it strides over
// the screened fragments).
cudaError_t run_pass_blocks(int prec, int cap, bool site, bool grain, int* blocks)
{
    int dev = 0, sms = 0, per_sm = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (e == cudaSuccess)
        e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, run_kernel(site ? 0 : prec, site, grain), 128,
                                                          phase_smem_bytes(cap, site));
    *blocks = std::max(1, sms * std::max(per_sm, 1));
    return e;
}

// Blocks of the small-fragment pass: as many as fit on the GPU at once (the
// grouped pass strides over its lists; the one-thread-per-fragment pass is a
// persistent grid whose warps split the phase's fragments).
cudaError_t small_pass_blocks(int prec, bool grain, int lane, int* blocks)
{
    int dev = 0, sms = 0, per_sm = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (e == cudaSuccess) {
        if (lane == LANE_PERSISTENT)
            e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, lane_kernel(grain), LANE_THREADS, 0);
        else
            e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, small_kernel(prec, grain), 128, 0);
    }
    *blocks = std::max(1, sms * std::max(per_sm, 1));
    return e;
}

// One window of the colour-phase path: set-up, then screen and run for each of
// the 8 phases.  Every argument is fixed for the batch (the window offset is
// read from wctl on the device), so the sequence can be captured in a graph.
// `sa.field` non-null selects the site-energy run pass (plain form),
// `sa.gbound` non-null the grain tables.
cudaError_t launch_window(int prec, const RepDesc* d_descs, int nrep, int64_t total_items,
                          unsigned long long* wctl, uint32_t* perms, ActEntry* act, int32_t* act_count,
                          uint8_t* cls, uint32_t* occ, VacRec* recs, int32_t* counts, int32_t* tracer,
                          unsigned long long* stats, uint32_t* status, int cap, int run_blocks,
                          int small_blocks, bool split_pass, int lane_form, const SiteArgs& sa, cudaStream_t st,
                          cudaStream_t side, cudaEvent_t fork, cudaEvent_t join)
{
    if (total_items <= 0) return cudaSuccess;
    const bool site = sa.field != nullptr, grain = sa.gbound != nullptr;
    k_window_setup<<<(nrep + 255) / 256, 256, 0, st>>>(d_descs, nrep, wctl, perms, act_count);
    const int64_t sblocks = (total_items + 255) / 256;
    const size_t smem = phase_smem_bytes(cap, site);
    const RunFn run = run_kernel(site ? 0 : prec, site, grain);
    const int lane = split_pass && !site && prec == 1 ? lane_form : LANE_NONE;
    const int split = !split_pass || site ? 0 : (lane == LANE_REGISTERS ? 2 : (lane == LANE_NONE ? 1 : 0));
    const SmallFn small = small_kernel(prec, grain);
    const LaneFn lanek = lane_kernel(grain);
    const LaneRegFn lanereg = grain ? k_run_lane_reg<true> : k_run_lane_reg<false>;
    for (int p = 0; p < 8; ++p) {
        if (lane == LANE_PERSISTENT) {  // every fragment of the colour; the dense ones listed for the warp pass after it
            lanek<<<small_blocks, LANE_THREADS, 0, st>>>(d_descs, nrep, total_items, p, wctl, perms, act, act_count,
                                                        occ, recs, counts, tracer, stats, status, cap, sa.gbound);
        } else if (site || prec == 0) {
            k_screen<0><<<(unsigned)sblocks, 256, 0, st>>>(d_descs, nrep, total_items, p, wctl, perms, counts, act,
                                                           act_count, split, cls);
        } else {
            k_screen<1><<<(unsigned)sblocks, 256, 0, st>>>(d_descs, nrep, total_items, p, wctl, perms, counts, act,
                                                           act_count, split, cls);
        }
        if (split) {  // the small-fragment pass and the general one touch disjoint fragments: side by side
            cudaError_t e = cudaEventRecord(fork, st);
            if (e == cudaSuccess) e = cudaStreamWaitEvent(side, fork, 0);
            if (e != cudaSuccess) return e;
            if (split == 1)
                small<<<small_blocks, 128, 0, side>>>(d_descs, act, total_items, act_count, p, wctl, occ, recs,
                                                      counts, tracer, stats, status, cap, sa.gbound);
            else
                lanereg<<<(unsigned)((total_items + 127) / 128), 128, 0, side>>>(
                    d_descs, nrep, total_items, p, wctl, perms, cls, occ, recs, counts, tracer, stats, status, cap,
                    sa.gbound);
            e = cudaEventRecord(join, side);
            if (e != cudaSuccess) return e;
        }
        run<<<run_blocks, 128, smem, st>>>(d_descs, act, act_count, p, wctl, occ, recs, counts, tracer, stats, status,
                                           cap, sa);
        if (split) {
            const cudaError_t e = cudaStreamWaitEvent(st, join, 0);
            if (e != cudaSuccess) return e;
        }
    }
    return cudaGetLastError();
}

cudaError_t launch_init_dopants(const RepDesc& D, int b_bits, int64_t n_fe, uint8_t* fe, cudaStream_t st)
{
    if (n_fe <= 0) return cudaSuccess;
    const int threads = 256;
    k_init_dopants<<<(unsigned)((n_fe + threads - 1) / threads), threads, 0, st>>>(D, b_bits, n_fe, fe);
    return cudaGetLastError();
}

// E_site of every O site of the batch from scratch: zero, then the vacancies'
// and the dopants' shell energies scattered with integer atomics.
cudaError_t launch_site_field(const RepDesc* d_descs, int nrep, const VacRec* recs, const int32_t* counts,
                              int64_t nfrag_total, int cap, int64_t nsite_total, const uint8_t* fe,
                              const SiteOff* bo, int n_bo, const SiteArgs& sa, cudaStream_t st)
{
    cudaError_t e = cudaMemsetAsync(sa.field, 0, sizeof(int32_t) * nsite_total, st);
    if (e != cudaSuccess) return e;
    const int threads = 256;
    if (sa.n_vv > 0) {
        const int64_t blocks = std::min<int64_t>(65536, (nfrag_total * cap + threads - 1) / threads);
        k_field_vac<<<(unsigned)std::max<int64_t>(blocks, 1), threads, 0, st>>>(d_descs, nrep, recs, counts,
                                                                              nfrag_total, cap, sa);
    }
    if (fe && n_bo > 0) {
        const int64_t ncell = nsite_total / 3;
        const int64_t blocks = std::min<int64_t>(65536, (ncell + threads - 1) / threads);
        k_field_dopant<<<(unsigned)std::max<int64_t>(blocks, 1), threads, 0, st>>>(d_descs, nrep, fe, ncell, bo,
                                                                                 n_bo, sa.field);
    }
    return cudaGetLastError();
}

cudaError_t launch_moments(const RepDesc& D, int species, const uint32_t* occ, const VacRec* recs,
                           const int32_t* counts, const int32_t* tracer, int cap,
                           unsigned long long* out, cudaStream_t st)
{
    cudaError_t e = cudaMemsetAsync(out, 0, 7 * sizeof(unsigned long long), st);
    if (e != cudaSuccess) return e;
    const int threads = 256;
    if (species == SP_V) {
        const int64_t nfrag = (int64_t)D.nf[0] * D.nf[1] * D.nf[2];
        int64_t blocks = (nfrag * cap + threads - 1) / threads;
        if (blocks > 4096) blocks = 4096;
        k_moments_vac<<<(unsigned)blocks, threads, 0, st>>>(recs, counts, D.frag_base, nfrag, cap, out);
    } else {
        int64_t blocks = (D.nsite + threads - 1) / threads;
        if (blocks > 4096) blocks = 4096;
        k_moments_ion<<<(unsigned)blocks, threads, 0, st>>>(D, occ, tracer, species, out);
    }
    return cudaGetLastError();
}

cudaError_t launch_moments_all(const RepDesc* d_descs, int nrep, const VacRec* recs, const int32_t* counts,
                               int64_t max_frag_per_replica, int cap, unsigned long long* out, cudaStream_t st)
{
    cudaError_t e = cudaMemsetAsync(out, 0, 7 * sizeof(unsigned long long) * nrep, st);
    if (e != cudaSuccess) return e;
    const int64_t per_block = (int64_t)MOM_THREADS * MOM_SLOTS_PER_THREAD;
    const int64_t chunks = std::max<int64_t>(1, (max_frag_per_replica * cap + per_block - 1) / per_block);
    dim3 grid((unsigned)chunks, (unsigned)nrep);
    k_moments_vac_all<<<grid, MOM_THREADS, 0, st>>>(d_descs, recs, counts, cap, out);
    return cudaGetLastError();
}

}  // namespace fkmc
