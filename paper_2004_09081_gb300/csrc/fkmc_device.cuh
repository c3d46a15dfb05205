// fkmc_device.cuh -- device-side definitions of the fragment kMC library:
// replica descriptors, Philox4x64-10, the two series logarithms that feed
// the residence-time clock (Eq. TimeStep of arXiv:2004.09081), the O-sublattice
// geometry and the fragment partition.
//
// Every floating-point operation in this file is written as an explicit
// round-to-nearest intrinsic (__dadd_rn, __fmul_rn, ...) so that no
// multiply-add is fused and each result is one IEEE operation in the order
// written.
#pragma once
#include <cstdint>

namespace fkmc {

constexpr int SP_O = 0, SP_H = 1, SP_V = 2;
constexpr uint32_t PURPOSE_INIT = 1u, PURPOSE_PERM = 2u, PURPOSE_HOP = 3u, PURPOSE_DOPE = 5u;
constexpr uint32_t PURPOSE_PICK = 6u, PURPOSE_NULL = 7u, PURPOSE_GRAIN = 8u;
constexpr uint32_t STATUS_OVERFLOW = 1u, STATUS_TIMEOUT = 2u, STATUS_EVENT_LIMIT = 4u, STATUS_ENERGY_RANGE = 8u;
// Hard bound on the events one fragment may execute in one colour phase
// (about 2.5e5 x the expected count at n_tau <= 64); reaching it ends the
// phase and reports an error instead of running on.
constexpr uint64_t MAX_EVENTS_PER_PHASE = 1ull << 24;

// One vacancy record: site key (t<<48 | z<<32 | y<<16 | x, so that key order
// is linear site order), unwrapped displacement in units of a/2, id.
struct __align__(8) VacRec {
    uint64_t key;
    int32_t d[3];
    uint32_t id;
};
static_assert(sizeof(VacRec) == 24, "record layout");

// Per-replica descriptor (device copy is read-only inside kernels).
struct RepDesc {
    int32_t L[3];          // cells per dimension
    int32_t nf[3];         // fragments per dimension (1 or even)
    int32_t base[3];       // L / nf
    int32_t rem[3];        // L % nf: the first `rem` fragments are one cell longer
    int32_t row_words;     // 32-bit words per occupancy row (16 sites per word)
    int32_t F;             // fixed-point fraction bits (mixed form)
    int32_t items;         // work items per colour phase = prod ceil(nf/2)
    uint32_t replica;
    int64_t items_off;     // prefix of `items` over replicas
    int64_t frag_base;     // first fragment of this replica in batch-wide arrays
    int64_t occ_word_off;  // first occupancy word of this replica
    int64_t site_off;      // first site of this replica (tracer field)
    int64_t nsite;
    uint64_t seed;
    uint64_t window;       // windows completed before the current run
    double k64[6];         // FP64 rate table, index 3*h + dz + 1
    uint64_t q[6];         // fixed-point rate table
    double tau;            // window length (s), plain clock
    double theta_tau;      // window length in units of 1/k32max, mixed clock
    double two_pow_F;      // 2^F, exact
    int32_t resident;      // 1: this replica runs in the replica-resident kernel
    int32_t pre_g;         // replica-resident kernel: colour phases whose first draws are made in one batch (1, 2, 4 or 8)
    int64_t btab_off;      // site energies: first Boltzmann-table entry of this replica
    int32_t bhi_mid;       // index of the high-table entry for m1 = 0
    int32_t bhi_len;       // entries of the high table
    // atom-based fragment kMC with null events (Sec. II.B)
    int64_t vac_off;       // first vacancy of this replica in the id-ordered array
    int64_t null_nv;       // vacancies (the atoms)
    int64_t null_nfrg;     // picks per step, min(N_frg, null_nv)
    int64_t pick_off;      // first pick of this replica in the batch-wide pick array
    uint64_t null_step;    // steps completed before the current call
    uint64_t qn[6];        // fixed-point rates, F_null = 63 - ceil(log2(8 null_nv))
    double two_pow_Fn;     // 2^F_null
    // grains: hops touching a boundary cell use these tables (type index - 6)
    double k64g[6];
    uint64_t qg[6];
    uint64_t qng[6];
    int32_t pre_ev;        // replica-resident kernel: events per fragment drawn in the batch (2: block 0; 4: blocks 0, 1)
    int32_t pad_ev_;
};

// One pick of the null-event form: the vacancy (by id) and its event (-1: null).
struct NullProp {
    int64_t v;
    int32_t n;
    int32_t pad;
};

// ---------------------------------------------------------------- site energies
// Interaction shells of the dopant/defect section of the paper: an O site's
// energy is a sum of pair energies (integers in units of 1e-4 eV) over the
// vacancies and dopants at the listed squared distances.  SiteOff is one
// partner position: site type t2 in the cell offset dc, energy e.
struct SiteOff {
    int8_t t2;
    int8_t dc[3];
    int32_t e;
};
constexpr int SITE_MAX_VV = 256;  // O partners of one O site inside the V-V shells
constexpr int SITE_MAX_BO = 512;  // O sites inside the V-dopant shells of one B site
constexpr int BOLTZ_LO = 512;     // Boltzmann factor of m units = hi[m >> 9] * lo[m & 511]

// Kernel arguments of the site-energy path (fixed for a batch).
struct SiteArgs {
    const SiteOff* vv;    // [3][SITE_MAX_VV] offsets by site type of the centre
    const double* btab;   // per replica: lo[BOLTZ_LO] then hi[bhi_len]
    int32_t* field;       // E_site of every O site (batch-wide site index)
    int32_t n_vv;         // offsets per site type
    int32_t e_self;       // energy of the a/sqrt2 shell: a hop partner's share of its target
    const uint8_t* gbound;  // grains: 1 per boundary cell (batch-wide cell index), or null
    const int32_t* g_elec;  // electrostatics: [replica][3][8] own-potential share of a hop, or null
};

// cell of a site, batch-wide index (a replica's cells start at site_off / 3)
__device__ __forceinline__ int64_t cell_index(const RepDesc& D, int x, int y, int z)
{
    return D.site_off / 3 + ((int64_t)z * D.L[1] + y) * D.L[0] + x;
}

// ---------------------------------------------------------------- Philox
// Philox4x64-10 (Salmon, Moraes, Dror, Shaw, SC'11): ten rounds of the
// multiply S-box on words 0 and 2 with the two published multipliers, Weyl
// key increments (golden ratio, sqrt(3)-1) between rounds.
struct U64x4 {
    uint64_t x[4];
};

__device__ __forceinline__ U64x4 philox4x64(uint64_t c0, uint64_t c1, uint64_t c2, uint64_t c3,
                                             uint64_t k0, uint64_t k1)
{
    const uint64_t M0 = 0xD2E7470EE14C6C93ull, M1 = 0xCA5A826395121157ull;
    const uint64_t W0 = 0x9E3779B97F4A7C15ull, W1 = 0xBB67AE8584CAA73Bull;
#pragma unroll
    for (int r = 0; r < 10; ++r) {
        const uint64_t hi0 = __umul64hi(M0, c0), lo0 = M0 * c0;
        const uint64_t hi1 = __umul64hi(M1, c2), lo1 = M1 * c2;
        const uint64_t n0 = hi1 ^ c1 ^ k0, n2 = hi0 ^ c3 ^ k1;
        c0 = n0; c1 = lo1; c2 = n2; c3 = lo0;
        k0 += W0; k1 += W1;
    }
    U64x4 o;
    o.x[0] = c0; o.x[1] = c1; o.x[2] = c2; o.x[3] = c3;
    return o;
}

__device__ __forceinline__ uint64_t key_word(uint32_t replica, uint32_t purpose)
{
    return ((uint64_t)replica << 8) | purpose;
}

// ---------------------------------------------------------------- logs
// -ln u from the atanh series ln m = 2 (s + s^3/3 + s^5/5 + ...),
// s = (m-1)/(m+1), m in [sqrt(1/2), sqrt(2)) (Abramowitz & Stegun 4.1.27),
// with u = m 2^e.

// ln 2 split for an exact e * LN2_HI (|e| < 2^20): ln 2 rounded to 32
// fraction bits, and the double nearest the remainder.
constexpr double LN2_HI = 0x1.62e42ff000000p-1;
constexpr double LN2_LO = -0x1.718432a1b0e26p-35;

// FP64 form: u = (2 floor(x/2^12) + 1) 2^-53, exactly representable in (0,1).
// With f = m - 1 (exact), s = f/(2+f), Q = s^2 (2/3 + 2 s^2/5 + ...), the
// identity 2s = f - f^2/2 + s f^2/2 gives ln m = f - (f^2/2 - s (f^2/2 + Q)):
// the exact f carries the result, rounding enters through the small terms;
// the final sum is ordered as in the classic fdlibm log (Sun, 1993).  Within
// 1 ulp of the correctly rounded -ln u.
__device__ __forceinline__ double neglog64(uint64_t x)
{
    const double u = __dmul_rn(__ull2double_rn(2ull * (x >> 12) + 1ull), 0x1p-53);
    const uint64_t bits = (uint64_t)__double_as_longlong(u);
    int e = (int)((bits >> 52) & 0x7ffull) - 1022;
    double m = __longlong_as_double((long long)((bits & 0x000fffffffffffffull) | 0x3fe0000000000000ull));
    if (m < 0.70710678118654752440) {
        m = __dmul_rn(m, 2.0);
        e -= 1;
    }
    const double f = __dsub_rn(m, 1.0);
    const double s = __ddiv_rn(f, __dadd_rn(2.0, f));
    const double s2 = __dmul_rn(s, s);
    double p = 2.0 / 21.0;
    p = __dadd_rn(2.0 / 19.0, __dmul_rn(s2, p));
    p = __dadd_rn(2.0 / 17.0, __dmul_rn(s2, p));
    p = __dadd_rn(2.0 / 15.0, __dmul_rn(s2, p));
    p = __dadd_rn(2.0 / 13.0, __dmul_rn(s2, p));
    p = __dadd_rn(2.0 / 11.0, __dmul_rn(s2, p));
    p = __dadd_rn(2.0 / 9.0, __dmul_rn(s2, p));
    p = __dadd_rn(2.0 / 7.0, __dmul_rn(s2, p));
    p = __dadd_rn(2.0 / 5.0, __dmul_rn(s2, p));
    p = __dadd_rn(2.0 / 3.0, __dmul_rn(s2, p));
    const double Q = __dmul_rn(s2, p);
    const double hfsq = __dmul_rn(__dmul_rn(0.5, f), f);
    const double de = __int2double_rn(e);
    const double inner = __dadd_rn(__dmul_rn(s, __dadd_rn(hfsq, Q)), __dmul_rn(de, LN2_LO));
    const double ln_u = __dsub_rn(__dmul_rn(de, LN2_HI), __dsub_rn(__dsub_rn(hfsq, inner), f));
    return -ln_u;
}

// FP32 form over the full 64-bit range: the leading one of (x|1) gives the
// binary exponent, the next 22 bits and a forced midpoint bit the mantissa.
__device__ __forceinline__ float neglog32(uint64_t x)
{
    x |= 1ull;
    const int lz = __clzll((long long)x);
    const int p = 63 - lz;
    const uint64_t nx = x << lz;
    const uint32_t mant = (uint32_t)(nx >> 40) | 1u;
    float m = __fmul_rn(__uint2float_rn(mant), 0x1p-23f);
    int e = p - 64;
    if (m > 1.41421356f) {
        m = __fmul_rn(m, 0.5f);
        e += 1;
    }
    const float s = __fdiv_rn(__fsub_rn(m, 1.0f), __fadd_rn(m, 1.0f));
    const float s2 = __fmul_rn(s, s);
    float q = 2.0f / 9.0f;
    q = __fadd_rn(2.0f / 7.0f, __fmul_rn(s2, q));
    q = __fadd_rn(2.0f / 5.0f, __fmul_rn(s2, q));
    q = __fadd_rn(2.0f / 3.0f, __fmul_rn(s2, q));
    q = __fadd_rn(2.0f, __fmul_rn(s2, q));
    const float lnm = __fmul_rn(s, q);
    const float ln_u = __fadd_rn(__fmul_rn(__int2float_rn(e), 0.693147182f), lnm);
    return -ln_u;
}

// A fragment that the screen pass of a colour phase keeps for the run pass,
// with the first Philox block of its phase (events 0 and 1).
struct ActEntry {
    int32_t rep;        // replica index in the batch
    int32_t nv;         // the fragment's vacancy count (unchanged until its run pass: hops leave a
                        // fragment only for fragments of other colours)
    int64_t fid;        // fragment index inside the replica
    uint64_t xs[2];     // selection words of events 0, 1
    uint64_t E[2];      // their exponential variates: fp64 bits (plain) or fp32 bits (mixed)
};
static_assert(sizeof(ActEntry) == 48, "active entry layout");

// Colour order of window w as 8 nibbles (nibble p = colour of phase p):
// Fisher-Yates shuffle of 0..7, j = mulhi(y_k, i+1), y_0..y_7 = Philox blocks (w,0), (w,1).
__device__ __forceinline__ uint32_t colour_perm_packed(uint64_t seed, uint32_t replica, uint64_t w)
{
    const U64x4 b0 = philox4x64(w, 0, 0, 0, seed, key_word(replica, PURPOSE_PERM));
    const U64x4 b1 = philox4x64(w, 1, 0, 0, seed, key_word(replica, PURPOSE_PERM));
    const uint64_t y[8] = {b0.x[0], b0.x[1], b0.x[2], b0.x[3], b1.x[0], b1.x[1], b1.x[2], b1.x[3]};
    uint32_t perm = 0x76543210u;
#pragma unroll
    for (int i = 7; i >= 1; --i) {
        const int j = (int)__umul64hi(y[7 - i], (uint64_t)(i + 1));
        const uint32_t pi = (perm >> (4 * i)) & 15u, pj = (perm >> (4 * j)) & 15u;
        perm &= ~((15u << (4 * i)) | (15u << (4 * j)));
        perm |= (pj << (4 * i)) | (pi << (4 * j));
    }
    return perm;
}

// ---------------------------------------------------------------- geometry
// Neighbour table in constant memory, filled by the host at load time:
// for site type t and neighbour n (ascending (dx,dy,dz)): packed
// {t2, dcx, dcy, dcz, dx, dy, dz} as signed bytes in two words.
struct NbEntry {
    int8_t t2, dc[3], d[3], pad;
};
struct NbTable {
    NbEntry e[3][8];
};

__device__ __forceinline__ int wrapc(int c, int L)
{
    return c < 0 ? c + L : (c >= L ? c - L : c);
}

__device__ __forceinline__ int frag_start(int i, int base, int rem)
{
    return i * base + min(i, rem);
}

__device__ __forceinline__ int frag_of(int c, int base, int rem)
{
    const int big = rem * (base + 1);
    return c < big ? c / (base + 1) : rem + (c - big) / base;
}

__device__ __forceinline__ uint64_t make_key(int t, int x, int y, int z)
{
    return ((uint64_t)t << 48) | ((uint64_t)z << 32) | ((uint64_t)y << 16) | (uint64_t)x;
}

__device__ __forceinline__ void split_key(uint64_t k, int& t, int& x, int& y, int& z)
{
    x = (int)(k & 0xffff);
    y = (int)((k >> 16) & 0xffff);
    z = (int)((k >> 32) & 0xffff);
    t = (int)(k >> 48);
}

// Occupancy layout: 2 bits per site, 16 sites of one row and type per word;
// the three site types' words of the same 16 cells are adjacent, then the
// row's next 16 cells, rows ordered (z, y), each row row_words groups long.
// A vacancy's 8 neighbours (the other two types, in its own row and the
// adjacent y and z rows) then lie in about three 32-byte sectors.
__host__ __device__ __forceinline__ int64_t occ_index(int64_t row_words, int L1, int t, int x, int y, int z)
{
    return (((int64_t)z * L1 + y) * row_words + (x >> 4)) * 3 + t;
}

// word index (within the batch occupancy array) and bit shift of a site
__device__ __forceinline__ int64_t occ_word(const RepDesc& D, int t, int x, int y, int z)
{
    return D.occ_word_off + occ_index(D.row_words, D.L[1], t, x, y, z);
}

__device__ __forceinline__ int occ_shift(int x) { return (x & 15) * 2; }

// Colour processed in `phase` of window w: Fisher-Yates shuffle of 0..7 with
// j = mulhi(y_k, i+1), y_0..y_7 = Philox blocks (w,0) and (w,1).
__device__ __forceinline__ int colour_of_phase(uint64_t seed, uint32_t replica, uint64_t w, int phase,
                                               int lane)
{
    const U64x4 blk = philox4x64(w, (uint64_t)(lane & 1), 0, 0, seed, key_word(replica, PURPOSE_PERM));
    uint32_t perm = 0x76543210u;  // nibble i holds perm[i]
#pragma unroll
    for (int i = 7; i >= 1; --i) {
        const int k = 7 - i;
        const uint64_t mine = blk.x[k & 3];
        const uint64_t y = __shfl_sync(0xffffffffu, mine, k >> 2);
        const int j = (int)__umul64hi(y, (uint64_t)(i + 1));
        const uint32_t pi = (perm >> (4 * i)) & 15u, pj = (perm >> (4 * j)) & 15u;
        perm &= ~((15u << (4 * i)) | (15u << (4 * j)));
        perm |= (pj << (4 * i)) | (pi << (4 * j));
    }
    return (int)((perm >> (4 * phase)) & 15u);
}

}  // namespace fkmc
