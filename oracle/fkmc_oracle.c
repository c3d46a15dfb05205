/*
 * fkmc_oracle.c -- serial CPU oracle for the windowed fragment kMC of
 * H. Nakata, "Development of a fragment kinetic Monte Carlo method for
 * efficient prediction of ionic diffusion in perovskite crystals"
 * (arXiv:2004.09081).
 *
 * TEST INFRASTRUCTURE ONLY.  This file is the slow, obviously correct
 * statement of what the GPU path computes.  Only the test-suite, the smoke
 * check and the CPU-baseline leg of the benchmark may load it.  It shares no
 * code, header, table or constant generator with the CUDA library: every
 * definition below (Philox, logarithms, geometry, partition, rates) is written
 * here from its published definition or from the paper.
 *
 * Compile with -O2 -ffp-contract=off (no fused multiply-add: every floating
 * point operation below is one IEEE round-to-nearest operation, in the order
 * written).
 *
 * What is computed (section / equation of the paper):
 *   - hop rates k = A exp(-Ea/(kB T))                 Sec. II.A, Eq. (RateCnst1)
 *     with the electrostatic shift of Sec. III (Ea -> Ea + dE_pot/2, z-projected)
 *   - event selection by cumulative rate              Sec. II.A, Eq. (eventSelection)
 *   - residence-time clock t += -ln(r')/sum k          Sec. II.A, Eq. (TimeStep)
 *   - fragment-local selection (p_i depends only on the
 *     rates inside the fragment once the clock is shared) Sec. II.B, Eq. (AtomP)
 *   - D from tracked trajectories                     Sec. III (per-atom tracking)
 *   - site-energy interactions (vacancy-vacancy and vacancy-dopant pair
 *     energies by coordination shell, barrier Ea + dE_site/2)
 *                                                    Sec. "Oxygen vacancy diffusion
 *                                                    with dopant and defect
 *                                                    interaction", Table add01
 *   - the atom-based fragment kMC with null events    Sec. II.B, Eqs. (AtomP),
 *     (vacancies as the atoms, N_frg picks per step)   (TimeStepFrg)
 *   - Voronoi grains whose boundary layer raises the   Sec. "Oxygen diffusion in
 *     barrier of every hop touching it (0.2 eV)          mu-scale BaTiO3 model"
 * The spatial fragments, checkerboard colour phases, synchronisation windows
 * and hand-off of boundary hops are the synchronous-sublattice reading of the
 * fragment scheme; every step is written out in fkmc_phase() below.
 *
 * Parity pins (tests/test_oracle_*.py): Philox against numpy's independent
 * Philox4x64-10, logarithms against libm, geometry against a brute-force
 * distance search, the single-vacancy closed forms D = Gamma d^2/6 and the
 * field drift, conservation laws, first-hop uniformity and agreement with
 * the conventional (non-fragmented) BKL of Sec. II.A.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define SP_O 0
#define SP_H 1
#define SP_V 2

#define PURPOSE_INIT 1u
#define PURPOSE_PERM 2u
#define PURPOSE_HOP 3u
#define PURPOSE_BKL 4u
#define PURPOSE_DOPE 5u
#define PURPOSE_PICK 6u
#define PURPOSE_NULL 7u
#define PURPOSE_GRAIN 8u

/* ------------------------------------------------------------------ */
/* Philox4x64-10 (Salmon, Moraes, Dror, Shaw, "Parallel random numbers:
 * as easy as 1, 2, 3", SC'11).  Counter c[4], key k[2]; ten rounds of
 * the S-box (multiply-high / multiply-low by M0 on c0 and M1 on c2), with
 * the Weyl key schedule (golden ratio and sqrt(3)-1 increments).        */
/* ------------------------------------------------------------------ */
void orc_philox4x64(const uint64_t ctr[4], const uint64_t key[2], uint64_t out[4])
{
    const uint64_t M0 = 0xD2E7470EE14C6C93ull, M1 = 0xCA5A826395121157ull;
    const uint64_t W0 = 0x9E3779B97F4A7C15ull, W1 = 0xBB67AE8584CAA73Bull;
    uint64_t x0 = ctr[0], x1 = ctr[1], x2 = ctr[2], x3 = ctr[3];
    uint64_t k0 = key[0], k1 = key[1];
    for (int r = 0; r < 10; r++) {
        unsigned __int128 p0 = (unsigned __int128)M0 * x0;
        unsigned __int128 p1 = (unsigned __int128)M1 * x2;
        uint64_t hi0 = (uint64_t)(p0 >> 64), lo0 = (uint64_t)p0;
        uint64_t hi1 = (uint64_t)(p1 >> 64), lo1 = (uint64_t)p1;
        x0 = hi1 ^ x1 ^ k0;
        x1 = lo1;
        x2 = hi0 ^ x3 ^ k1;
        x3 = lo0;
        k0 += W0;
        k1 += W1;
    }
    out[0] = x0; out[1] = x1; out[2] = x2; out[3] = x3;
}

static uint64_t mulhi64(uint64_t a, uint64_t b)
{
    return (uint64_t)(((unsigned __int128)a * b) >> 64);
}

static void key_for(uint64_t seed, uint32_t replica, uint32_t purpose, uint64_t key[2])
{
    key[0] = seed;
    key[1] = ((uint64_t)replica << 8) | purpose;
}

/* ------------------------------------------------------------------ */
/* Natural logarithm from its series: with u = m 2^e, m in [sqrt(1/2),
 * sqrt(2)), ln u = e ln2 + 2 atanh(s), s = (m-1)/(m+1), and
 * 2 atanh(s) = 2 (s + s^3/3 + s^5/5 + ...)  (Abramowitz & Stegun 4.1.27).
 * Both clocks of the method draw their exponential variates through
 * these two functions.                                                  */
/* ------------------------------------------------------------------ */

/* ln 2 split so that e * LN2_HI is exact for |e| < 2^20: LN2_HI is ln 2
 * rounded to 32 fraction bits, LN2_LO the double nearest ln 2 - LN2_HI. */
static const double LN2_HI = 0x1.62e42ff000000p-1;
static const double LN2_LO = -0x1.718432a1b0e26p-35;

/* FP64: u = (2 floor(x/2^12) + 1) 2^-53, an exact double in (0,1). Returns -ln u.
 * With f = m - 1 (exact), s = f / (2 + f) and R = 2 s^3/3 + 2 s^5/5 + ... =
 * s Q, Q = s^2 (2/3 + 2 s^2/5 + ...), the identity 2 s = f - f^2/2 + s f^2/2
 * gives ln m = f - (f^2/2 - s (f^2/2 + Q)): the exact f carries the result and
 * rounding enters only through the smaller terms.  The order of the final sum
 * is that of the classic fdlibm log (Sun Microsystems, 1993); with it the
 * result is within 1 ulp of the correctly rounded -ln u. */
double orc_neglog64(uint64_t x)
{
    double u = (double)(2 * (x >> 12) + 1) * 0x1p-53;
    uint64_t bits;
    memcpy(&bits, &u, 8);
    int e = (int)((bits >> 52) & 0x7ff) - 1022;
    uint64_t mb = (bits & 0x000fffffffffffffull) | 0x3fe0000000000000ull;
    double m;
    memcpy(&m, &mb, 8); /* m in [0.5, 1) */
    if (m < 0.70710678118654752440) { m = m * 2.0; e = e - 1; }
    double f = m - 1.0;
    double s = f / (2.0 + f);
    double s2 = s * s;
    double p = 2.0 / 21.0;
    p = 2.0 / 19.0 + s2 * p;
    p = 2.0 / 17.0 + s2 * p;
    p = 2.0 / 15.0 + s2 * p;
    p = 2.0 / 13.0 + s2 * p;
    p = 2.0 / 11.0 + s2 * p;
    p = 2.0 / 9.0 + s2 * p;
    p = 2.0 / 7.0 + s2 * p;
    p = 2.0 / 5.0 + s2 * p;
    p = 2.0 / 3.0 + s2 * p;
    double Q = s2 * p;
    double hfsq = (0.5 * f) * f;
    double de = (double)e;
    double ln_u = de * LN2_HI - ((hfsq - (s * (hfsq + Q) + de * LN2_LO)) - f);
    return -ln_u;
}

/* orc_neglog64 of n inputs (for the accuracy pin over many points). */
void orc_neglog64_batch(const uint64_t* x, double* out, int64_t n)
{
    for (int64_t i = 0; i < n; i++) out[i] = orc_neglog64(x[i]);
}

/* FP32 with the full 64-bit range: the leading one of x (x|1) fixes the
 * binary exponent, the next 22 bits plus a forced midpoint bit the mantissa
 * m in [1,2).  Returns -ln u for u = m 2^(p-64), p the leading-one position. */
float orc_neglog32(uint64_t x)
{
    x |= 1ull;
    int lz = 0;
    while (!(x & (1ull << 63))) { x <<= 1; lz++; }
    int p = 63 - lz;
    uint32_t mant = (uint32_t)(x >> 40) | 1u; /* 24 bits, bit 23 set */
    float m = (float)mant * 0x1p-23f;
    int e = p - 64;
    if (m > 1.41421356f) { m = m * 0.5f; e = e + 1; }
    float s = (m - 1.0f) / (m + 1.0f);
    float s2 = s * s;
    float q = 2.0f / 9.0f;
    q = 2.0f / 7.0f + s2 * q;
    q = 2.0f / 5.0f + s2 * q;
    q = 2.0f / 3.0f + s2 * q;
    q = 2.0f + s2 * q;
    float lnm = s * q;
    float ln_u = (float)e * 0.693147182f + lnm;
    return -ln_u;
}

/* ------------------------------------------------------------------ */
/* Geometry of the O sublattice (Fig. 2): cubic cell of edge a, O at the
 * three face centres.  Site types t = 0,1,2 sit at a/2 * e_t from the cell
 * corner.  Positions are kept in units of a/2.  The 8 nearest neighbours
 * (distance a/sqrt2) are found by a brute-force distance search and listed in
 * ascending lexicographic order of the displacement (dx, dy, dz).       */
/* ------------------------------------------------------------------ */
typedef struct { int t2; int dc[3]; int d[3]; } orc_nb;
static orc_nb NB[3][8];
static int nb_ready = 0;

static int cmp_nb(const void* a, const void* b)
{
    const orc_nb* p = (const orc_nb*)a;
    const orc_nb* q = (const orc_nb*)b;
    for (int k = 0; k < 3; k++)
        if (p->d[k] != q->d[k]) return p->d[k] < q->d[k] ? -1 : 1;
    return 0;
}

static void build_neighbours(void)
{
    if (nb_ready) return;
    for (int t = 0; t < 3; t++) {
        int n = 0;
        orc_nb cand[81];
        for (int t2 = 0; t2 < 3; t2++)
            for (int cx = -1; cx <= 1; cx++)
                for (int cy = -1; cy <= 1; cy++)
                    for (int cz = -1; cz <= 1; cz++) {
                        int c[3] = {cx, cy, cz};
                        int d[3], r2 = 0;
                        for (int k = 0; k < 3; k++) {
                            d[k] = 2 * c[k] + (k == t2) - (k == t);
                            r2 += d[k] * d[k];
                        }
                        if (r2 != 2) continue;
                        cand[n].t2 = t2;
                        for (int k = 0; k < 3; k++) { cand[n].dc[k] = c[k]; cand[n].d[k] = d[k]; }
                        n++;
                    }
        qsort(cand, n, sizeof(orc_nb), cmp_nb);
        for (int i = 0; i < 8 && i < n; i++) NB[t][i] = cand[i];
        if (n != 8) { /* cannot happen for this lattice; leave table unusable */
            memset(NB[t], 0, sizeof(NB[t]));
        }
    }
    nb_ready = 1;
}

/* export of the neighbour table: out[t][n] = {t2, dcx, dcy, dcz, dx, dy, dz} */
void orc_neighbour_table(int32_t* out)
{
    build_neighbours();
    for (int t = 0; t < 3; t++)
        for (int n = 0; n < 8; n++) {
            int32_t* o = out + (t * 8 + n) * 7;
            o[0] = NB[t][n].t2;
            for (int k = 0; k < 3; k++) { o[1 + k] = NB[t][n].dc[k]; o[4 + k] = NB[t][n].d[k]; }
        }
}

/* ------------------------------------------------------------------ */
/* Lattice state                                                       */
/* ------------------------------------------------------------------ */
typedef struct {
    int64_t site;   /* linear index ((t*nz + z)*ny + y)*nx + x */
    int32_t d[3];   /* unwrapped vacancy displacement, units of a/2 */
    uint32_t id;
} orc_rec;

typedef struct {
    int n, cap;
    orc_rec* r;
} orc_list;

typedef struct {
    int L[3];       /* cells nx, ny, nz */
    int nf[3];      /* fragments per dimension (1 or even) */
    int64_t nsite;
    uint64_t seed;
    uint32_t replica;
    int tracer;
    uint8_t* occ;   /* species per site */
    int32_t* tdisp; /* tracer: ion displacement per site, 3 per site */
    int nfrag;
    orc_list* frag; /* vacancy records per fragment */
    /* rate tables */
    int precision;  /* 0 plain FP64, 1 mixed */
    double k64[6];
    float k32[6];
    uint64_t q[6];
    int F;
    double tau, theta_tau, k32max;
    int rates_set;
    double T;       /* temperature of the rate table (K) */
    /* grains: boundary cells raise the barrier of hops touching them */
    int grains_on;
    int32_t* grain;    /* grain of each cell, [z][y][x] */
    uint8_t* gbound;   /* 1 for a boundary cell */
    double gb_eV;      /* barrier added to a boundary hop */
    double k64g[6];    /* rate tables of boundary hops */
    float k32g[6];
    uint64_t qg[6];
    double rate_args[8]; /* Ea_O, Ea_H, A, q_O, q_H, T, Ez, a of the last set_rates */
    int rate_cap;
    double rate_ntau;
    /* site-energy interactions (plain form only) */
    int site_on;
    int elec_on;        /* electrostatic potential of the vacancy charges (frozen field) */
    int32_t* elec_u;    /* q phi of every O site, 1e-4 eV units */
    int32_t elec_g[3][8]; /* a hop's share of the vacancy's own potential, 1e-4 eV units */
    uint8_t* fe;    /* dopant (Fe) on the B site of each cell, [z][y][x] */
    int n_vv, n_fe; /* offsets to the O sites / B sites inside the energy shells */
    struct { int t2; int dc[3]; int32_t e; } vv[3][512];
    struct { int dc[3]; int32_t e; } feo[3][512];
    /* atom-based fragment kMC with null events (Sec. II.B) */
    uint64_t null_step;
    double theta_null; /* its clock in units of 1/k32max */
    int64_t* claimed;  /* per site: 1 + the step whose earlier pick claimed it */
    /* counters */
    uint64_t window;
    uint64_t hops;
    uint64_t handoffs;
    double clock_sum; /* sum over fragment phases of the final clock (diagnostic) */
} orc_lattice;

/* Fragments per dimension for a target edge e (the paper fixes neither; the
 * reading): the even count nearest L/e, ties to the larger, among the even
 * counts 2, 4, ... that keep every fragment at least 2 cells long (edges are
 * floor(L/n) or ceil(L/n)); one fragment when no even count does (L < 4). */
int orc_partition_count(int L, int e)
{
    if (L < 1 || e < 1) return 0;
    double target = (double)L / (double)e;
    int best = 1;
    double best_dist = 0.0;
    for (int n = 2; L / n >= 2; n += 2) {
        double dist = fabs((double)n - target);
        if (best == 1 || dist <= best_dist) {
            best = n;
            best_dist = dist;
        }
    }
    return best;
}

static int frag_start(int L, int nf, int i)
{
    int base = L / nf, rem = L % nf;
    return i * base + (i < rem ? i : rem);
}

static int frag_of_cell(int L, int nf, int c)
{
    int i = 0;
    while (frag_start(L, nf, i + 1) <= c) i++;
    return i;
}

static int64_t site_index(const orc_lattice* lat, int t, int x, int y, int z)
{
    return (((int64_t)t * lat->L[2] + z) * lat->L[1] + y) * lat->L[0] + x;
}

static void site_coords(const orc_lattice* lat, int64_t s, int* t, int c[3])
{
    c[0] = (int)(s % lat->L[0]); s /= lat->L[0];
    c[1] = (int)(s % lat->L[1]); s /= lat->L[1];
    c[2] = (int)(s % lat->L[2]); s /= lat->L[2];
    *t = (int)s;
}

static int wrap(int c, int L) { c %= L; return c < 0 ? c + L : c; }

static int64_t neighbour_site(const orc_lattice* lat, int64_t s, int n)
{
    int t, c[3];
    site_coords(lat, s, &t, c);
    const orc_nb* nb = &NB[t][n];
    return site_index(lat, nb->t2, wrap(c[0] + nb->dc[0], lat->L[0]),
                      wrap(c[1] + nb->dc[1], lat->L[1]), wrap(c[2] + nb->dc[2], lat->L[2]));
}

static int fragment_of_site(const orc_lattice* lat, int64_t s)
{
    int t, c[3];
    site_coords(lat, s, &t, c);
    int f[3];
    for (int k = 0; k < 3; k++) f[k] = frag_of_cell(lat->L[k], lat->nf[k], c[k]);
    return (f[2] * lat->nf[1] + f[1]) * lat->nf[0] + f[0];
}

static int fragment_colour(const orc_lattice* lat, int F)
{
    int fx = F % lat->nf[0], fy = (F / lat->nf[0]) % lat->nf[1], fz = F / (lat->nf[0] * lat->nf[1]);
    return (fx & 1) | ((fy & 1) << 1) | ((fz & 1) << 2);
}

static void list_push(orc_list* l, orc_rec r)
{
    if (l->n == l->cap) {
        l->cap = l->cap ? 2 * l->cap : 8;
        l->r = (orc_rec*)realloc(l->r, sizeof(orc_rec) * l->cap);
    }
    l->r[l->n++] = r;
}

/* ------------------------------------------------------------------ */
/* Initial placement: a keyed bijection of [0, nsite) (a 4-round balanced
 * Feistel network with cycle walking, Black & Rogaway, "Ciphers with
 * arbitrary finite domains", CT-RSA 2002; round function = Philox).
 * Particle i < n_vac is a vacancy with id i, the next n_H are H-.      */
/* ------------------------------------------------------------------ */
uint64_t orc_feistel(uint64_t i, uint64_t nsite, uint64_t seed, uint32_t replica)
{
    int b = 1;
    while (((uint64_t)1 << (2 * b)) < nsite) b++;
    uint64_t mask = ((uint64_t)1 << b) - 1;
    uint64_t key[2];
    key_for(seed, replica, PURPOSE_INIT, key);
    uint64_t v = i;
    do {
        uint64_t L = v >> b, R = v & mask;
        for (int k = 0; k < 4; k++) {
            uint64_t ctr[4] = {R, (uint64_t)k, 0, 0}, o[4];
            orc_philox4x64(ctr, key, o);
            uint64_t nl = R, nr = L ^ (o[0] & mask);
            L = nl; R = nr;
        }
        v = (L << b) | R;
    } while (v >= nsite);
    return v;
}

/* Colour order of window w: Fisher-Yates shuffle of (0..7) driven by two
 * Philox blocks, j = floor(y * (i+1) / 2^64).                          */
void orc_colour_perm(uint64_t seed, uint32_t replica, uint64_t w, int32_t perm[8])
{
    uint64_t key[2], y[8];
    key_for(seed, replica, PURPOSE_PERM, key);
    uint64_t c0[4] = {w, 0, 0, 0}, c1[4] = {w, 1, 0, 0};
    orc_philox4x64(c0, key, y);
    orc_philox4x64(c1, key, y + 4);
    for (int i = 0; i < 8; i++) perm[i] = i;
    for (int i = 7; i >= 1; i--) {
        int j = (int)mulhi64(y[7 - i], (uint64_t)(i + 1));
        int tmp = perm[i]; perm[i] = perm[j]; perm[j] = tmp;
    }
}

orc_lattice* orc_create(int nx, int ny, int nz, int nfx, int nfy, int nfz, int64_t n_vac,
                        int64_t n_H, uint64_t seed, uint32_t replica, int tracer)
{
    build_neighbours();
    int L[3] = {nx, ny, nz}, nf[3] = {nfx, nfy, nfz};
    for (int k = 0; k < 3; k++) {
        if (L[k] < 1 || nf[k] < 1 || nf[k] > L[k]) return NULL;
        if (nf[k] > 1 && ((nf[k] & 1) || L[k] / nf[k] < 2)) return NULL;
    }
    int64_t nsite = 3 * (int64_t)nx * ny * nz;
    if (n_vac < 0 || n_H < 0 || n_vac + n_H > nsite) return NULL;
    orc_lattice* lat = (orc_lattice*)calloc(1, sizeof(orc_lattice));
    memcpy(lat->L, L, sizeof L);
    memcpy(lat->nf, nf, sizeof nf);
    lat->nsite = nsite;
    lat->seed = seed;
    lat->replica = replica;
    lat->tracer = tracer;
    lat->occ = (uint8_t*)calloc((size_t)nsite, 1);
    if (tracer) lat->tdisp = (int32_t*)calloc((size_t)nsite * 3, sizeof(int32_t));
    lat->nfrag = nfx * nfy * nfz;
    lat->frag = (orc_list*)calloc((size_t)lat->nfrag, sizeof(orc_list));
    for (int64_t i = 0; i < n_vac + n_H; i++) {
        int64_t s = (int64_t)orc_feistel((uint64_t)i, (uint64_t)nsite, seed, replica);
        if (i < n_vac) {
            lat->occ[s] = SP_V;
            orc_rec r = {s, {0, 0, 0}, (uint32_t)i};
            list_push(&lat->frag[fragment_of_site(lat, s)], r);
        } else {
            lat->occ[s] = SP_H;
        }
    }
    return lat;
}

void orc_destroy(orc_lattice* lat)
{
    if (!lat) return;
    for (int f = 0; f < lat->nfrag; f++) free(lat->frag[f].r);
    free(lat->frag);
    free(lat->occ);
    free(lat->tdisp);
    free(lat->fe);
    free(lat->claimed);
    free(lat->grain);
    free(lat->gbound);
    free(lat->elec_u);
    free(lat);
}

/* ------------------------------------------------------------------ */
/* Rates, Eq. (RateCnst1) with the ESP term of Sec. III:
 *   k = A exp(-(Ea_h + dU/2) / (kB T)),  dU = -q_h E_z dz_V,
 * dz_V = dz * a/2 the vacancy's z displacement (the ion moves the other
 * way), R of the paper read as Boltzmann's constant in eV/K.  Table index
 * ty = 3*h + (dz+1), h = 0 for O<->V and 1 for H<->V.
 * Mixed form: k32 = fp32 rounding of k64; q = rint(k32/k32max * 2^F) with
 * F = 63 - ceil(log2(8 C_v)) so a fragment's exact sum stays below 2^63.
 * Window length tau = n_tau / (8 k_fast), k_fast the largest FP64 rate of
 * the species present (H- entries count only when the lattice holds H-).  */
/* ------------------------------------------------------------------ */
static const double KB_EV = 8.617333262e-5;

int orc_rate_table(double Ea_O, double Ea_H, double A, double q_O, double q_H, double T_K,
                   double Ez_Vpm, double a_ang, int cap_v, double* k64, float* k32,
                   uint64_t* q, int32_t* F_out)
{
    if (!(T_K > 0) || cap_v < 1) return -1;
    double Ea[2] = {Ea_O, Ea_H}, qc[2] = {q_O, q_H};
    double half_a_m = 0.5 * a_ang * 1e-10;
    for (int h = 0; h < 2; h++)
        for (int dz = -1; dz <= 1; dz++) {
            double dz_m = (double)dz * half_a_m;
            double dU = -(qc[h] * Ez_Vpm) * dz_m;
            double barrier = Ea[h] + 0.5 * dU;
            k64[3 * h + dz + 1] = A * exp(-(barrier / (KB_EV * T_K)));
        }
    float kmax = 0.0f;
    for (int i = 0; i < 6; i++) {
        k32[i] = (float)k64[i];
        if (k32[i] > kmax) kmax = k32[i];
    }
    int lg = 0;
    while (((int64_t)1 << lg) < 8 * (int64_t)cap_v) lg++;
    int F = 63 - lg;
    for (int i = 0; i < 6; i++) q[i] = (uint64_t)llrint(ldexp((double)k32[i] / (double)kmax, F));
    *F_out = F;
    return 0;
}

int orc_set_rates(orc_lattice* lat, double Ea_O, double Ea_H, double A, double q_O, double q_H,
                  double T_K, double Ez_Vpm, double a_ang, int cap_v, double n_tau, int precision)
{
    int32_t F;
    if (orc_rate_table(Ea_O, Ea_H, A, q_O, q_H, T_K, Ez_Vpm, a_ang, cap_v, lat->k64, lat->k32,
                       lat->q, &F))
        return -1;
    lat->F = F;
    int64_t nH = 0;
    for (int64_t s = 0; s < lat->nsite; s++) nH += lat->occ[s] == SP_H;
    double kmax = 0.0;
    float kmax32 = 0.0f;
    for (int i = 0; i < 6; i++) {
        if ((i < 3 || nH > 0) && lat->k64[i] > kmax) kmax = lat->k64[i];
        if (lat->k32[i] > kmax32) kmax32 = lat->k32[i];
    }
    if ((lat->site_on || lat->elec_on) && precision != 0) return -1;
    lat->T = T_K;
    {
        double a[8] = {Ea_O, Ea_H, A, q_O, q_H, T_K, Ez_Vpm, a_ang};
        memcpy(lat->rate_args, a, sizeof a);
        lat->rate_cap = cap_v;
        lat->rate_ntau = n_tau;
    }
    if (lat->grains_on) {
        /* boundary hops: the same table with both barriers raised by gb_eV; the
         * mixed form quantises them against the bulk table's k32max */
        int32_t Fg;
        float k32b[6];
        uint64_t qb[6];
        if (orc_rate_table(Ea_O + lat->gb_eV, Ea_H + lat->gb_eV, A, q_O, q_H, T_K, Ez_Vpm, a_ang, cap_v,
                           lat->k64g, k32b, qb, &Fg))
            return -1;
        float kmax = 0.0f;
        for (int i = 0; i < 6; i++) if (lat->k32[i] > kmax) kmax = lat->k32[i];
        for (int i = 0; i < 6; i++) {
            lat->k32g[i] = k32b[i];
            lat->qg[i] = (uint64_t)llrint(ldexp((double)k32b[i] / (double)kmax, F));
        }
    }
    lat->tau = n_tau / (8.0 * kmax);
    lat->k32max = (double)kmax32;
    lat->theta_tau = lat->tau * lat->k32max;
    lat->precision = precision;
    lat->rates_set = 1;
    return 0;
}

/* ------------------------------------------------------------------ */
/* Site-energy interactions (Sec. "Oxygen vacancy diffusion with dopant and
 * defect interaction"): the energy of a vacancy at site s is
 *   E_site(s) = sum over shells k of  N_VV,k(s) e_VV,k + N_VFe,k(s) e_VFe,k,
 * N counting the other vacancies (O sites) and the dopants (B sites, one per
 * cell at the cell corner) at the shell's distance from s.  A hop of the
 * vacancy from s to j has barrier Ea + dU/2 + (E_site(j) - E_site(s))/2,
 * E_site(j) counted without the moving vacancy itself (it is the energy
 * change of the whole configuration, so detailed balance holds).
 * Shells are named by their squared distance in units of (a/2)^2: O-O shells
 * are even (2 = a/sqrt2, 4 = a, 6, 8, 10, ...), O-B shells odd (1 = a/2, 5,
 * 9, 13, ...).  Energies are held as integers in units of 1e-4 eV
 * (rint(e * 1e4)), so every energy difference is exact.
 * The Boltzmann factor exp(-dE/(2 kB T)) of an energy difference of m units is
 * evaluated as exp(-(512 m1) c) * exp(-m0 c), m = 512 m1 + m0 with
 * 0 <= m0 < 512 and c = 1e-4 / (2 kB T); the rate is (k_table * first) *
 * second, each product one IEEE rounding.                              */
/* ------------------------------------------------------------------ */
static int32_t energy_quanta(double eV) { return (int32_t)llrint(eV * 1e4); }

void orc_place_dopants(orc_lattice* lat, int64_t n_fe)
{
    /* keyed bijection of the cell indices (same Feistel construction as the
     * vacancy placement, its own key): cells f(0..n_fe-1) hold a dopant */
    int64_t ncell = (int64_t)lat->L[0] * lat->L[1] * lat->L[2];
    free(lat->fe);
    lat->fe = (uint8_t*)calloc((size_t)ncell, 1);
    int b = 1;
    while (((uint64_t)1 << (2 * b)) < (uint64_t)ncell) b++;
    uint64_t mask = ((uint64_t)1 << b) - 1;
    uint64_t key[2];
    key_for(lat->seed, lat->replica, PURPOSE_DOPE, key);
    for (int64_t i = 0; i < n_fe && i < ncell; i++) {
        uint64_t v = (uint64_t)i;
        do {
            uint64_t Lh = v >> b, Rh = v & mask;
            for (int k = 0; k < 4; k++) {
                uint64_t ctr[4] = {Rh, (uint64_t)k, 0, 0}, o[4];
                orc_philox4x64(ctr, key, o);
                uint64_t nl = Rh, nr = Lh ^ (o[0] & mask);
                Lh = nl; Rh = nr;
            }
            v = (Lh << b) | Rh;
        } while (v >= (uint64_t)ncell);
        lat->fe[v] = 1;
    }
}

void orc_set_dopants(orc_lattice* lat, const uint8_t* cells)
{
    int64_t ncell = (int64_t)lat->L[0] * lat->L[1] * lat->L[2];
    free(lat->fe);
    lat->fe = (uint8_t*)malloc((size_t)ncell);
    for (int64_t c = 0; c < ncell; c++) lat->fe[c] = cells[c] ? 1 : 0;
}

int orc_get_dopants(const orc_lattice* lat, uint8_t* cells)
{
    int64_t ncell = (int64_t)lat->L[0] * lat->L[1] * lat->L[2];
    if (lat->fe) memcpy(cells, lat->fe, (size_t)ncell);
    else memset(cells, 0, (size_t)ncell);
    return 0;
}

/* Shell offsets by exhaustive search over a box of cells: every O site (or B
 * site) whose squared distance from a site of type t is one of the listed
 * shells.  n = 0 turns the interactions off. */
int orc_set_site_energy(orc_lattice* lat, int n_vv, const int32_t* vv_d2, const double* vv_eV,
                        int n_fe, const int32_t* fe_d2, const double* fe_eV)
{
    if (n_vv < 0 || n_vv > 8 || n_fe < 0 || n_fe > 8) return -1;
    if (n_vv == 0 && n_fe == 0) { lat->site_on = 0; lat->n_vv = lat->n_fe = 0; return 0; }
    if (lat->rates_set && lat->precision != 0) return -1;
    /* a shell distance beyond the search box is an error */
    for (int q = 0; q < n_vv; q++) if (vv_d2[q] <= 0 || vv_d2[q] > 36) return -1;
    for (int q = 0; q < n_fe; q++) if (fe_d2[q] <= 0 || fe_d2[q] > 36) return -1;
    int reach_vv = 0, reach_all = 0;
    int cnt_vv[3] = {0, 0, 0}, cnt_fe[3] = {0, 0, 0};
    int hit_vv[8] = {0}, hit_fe[8] = {0};
    for (int t = 0; t < 3; t++) {
        for (int cz = -4; cz <= 4; cz++)
            for (int cy = -4; cy <= 4; cy++)
                for (int cx = -4; cx <= 4; cx++) {
                    int c[3] = {cx, cy, cz};
                    /* O sites of type t2 in cell n + c */
                    for (int t2 = 0; t2 < 3; t2++) {
                        int r2 = 0;
                        for (int k = 0; k < 3; k++) {
                            int d = 2 * c[k] + (k == t2) - (k == t);
                            r2 += d * d;
                        }
                        for (int q = 0; q < n_vv; q++)
                            if (vv_d2[q] == r2) {
                                if (cnt_vv[t] == 512) return -1;
                                hit_vv[q] = 1;
                                lat->vv[t][cnt_vv[t]].t2 = t2;
                                for (int k = 0; k < 3; k++) lat->vv[t][cnt_vv[t]].dc[k] = c[k];
                                lat->vv[t][cnt_vv[t]].e = energy_quanta(vv_eV[q]);
                                cnt_vv[t]++;
                                for (int k = 0; k < 3; k++) {
                                    int a = c[k] < 0 ? -c[k] : c[k];
                                    if (a > reach_vv) reach_vv = a;
                                    if (a > reach_all) reach_all = a;
                                }
                            }
                    }
                    /* the B site at the corner of cell n + c */
                    int r2 = 0;
                    for (int k = 0; k < 3; k++) {
                        int d = 2 * c[k] - (k == t);
                        r2 += d * d;
                    }
                    for (int q = 0; q < n_fe; q++)
                        if (fe_d2[q] == r2) {
                            if (cnt_fe[t] == 512) return -1;
                            hit_fe[q] = 1;
                            for (int k = 0; k < 3; k++) lat->feo[t][cnt_fe[t]].dc[k] = c[k];
                            lat->feo[t][cnt_fe[t]].e = energy_quanta(fe_eV[q]);
                            cnt_fe[t]++;
                            for (int k = 0; k < 3; k++) {
                                int a = c[k] < 0 ? -c[k] : c[k];
                                if (a > reach_all) reach_all = a;
                            }
                        }
                }
    }
    /* a shell distance that the lattice does not have is an error */
    for (int q = 0; q < n_vv; q++) if (!hit_vv[q]) return -1;
    for (int q = 0; q < n_fe; q++) if (!hit_fe[q]) return -1;
    if (cnt_vv[0] != cnt_vv[1] || cnt_vv[0] != cnt_vv[2]) return -1;
    for (int k = 0; k < 3; k++) {
        /* every offset lands on a distinct site of the periodic lattice */
        if (lat->L[k] < 2 * reach_all + 1) return -1;
        /* same-colour fragments neither read nor write what the other reads:
         * reads reach 1 + reach_vv cells out of a fragment, writes 1 cell */
        if (lat->nf[k] > 1 && lat->L[k] / lat->nf[k] < 2 + reach_vv) return -1;
    }
    lat->n_vv = cnt_vv[0];
    lat->n_fe = cnt_fe[0];
    lat->site_on = 1;
    if (!lat->fe) lat->fe = (uint8_t*)calloc((size_t)lat->L[0] * lat->L[1] * lat->L[2], 1);
    return 0;
}

/* export of the shell offsets of site type t: rows {t2, dcx, dcy, dcz, e}
 * (V-V, t2 = the O site type) then rows {-1, dcx, dcy, dcz, e} (V-Fe) */
int orc_site_shells(const orc_lattice* lat, int t, int32_t* out, int max_rows)
{
    int k = 0;
    for (int i = 0; i < lat->n_vv && k < max_rows; i++, k++) {
        int32_t* o = out + 5 * k;
        o[0] = lat->vv[t][i].t2;
        for (int d = 0; d < 3; d++) o[1 + d] = lat->vv[t][i].dc[d];
        o[4] = lat->vv[t][i].e;
    }
    for (int i = 0; i < lat->n_fe && k < max_rows; i++, k++) {
        int32_t* o = out + 5 * k;
        o[0] = -1;
        for (int d = 0; d < 3; d++) o[1 + d] = lat->feo[t][i].dc[d];
        o[4] = lat->feo[t][i].e;
    }
    return k;
}

/* Electrostatics (the Poisson-solved potential of the mu-scale model, with
 * the vacancy charges as its source): a frozen field u(s) = rint(q phi(s) 1e4)
 * joins E_site, and a hop s -> j (neighbour n of a type-t site) leaves out the
 * vacancy's own potential: its energy difference loses g[t][n] =
 * rint(q^2 (G(j, s) - G(s, s)) 1e4).  u and g are inputs (oracle/poisson.py
 * computes them); NULL u turns the term off. */
int orc_set_elec(orc_lattice* lat, const int32_t* u, const int32_t* g)
{
    if (!u) { lat->elec_on = 0; return 0; }
    if (lat->rates_set && lat->precision != 0) return -1;
    free(lat->elec_u);
    lat->elec_u = (int32_t*)malloc(sizeof(int32_t) * (size_t)lat->nsite);
    memcpy(lat->elec_u, u, sizeof(int32_t) * (size_t)lat->nsite);
    memcpy(lat->elec_g, g, sizeof(lat->elec_g));
    lat->elec_on = 1;
    return 0;
}

/* E_site of site s in energy units, the site `exclude` counted as empty */
int64_t orc_site_energy(const orc_lattice* lat, int64_t s, int64_t exclude)
{
    if (!lat->site_on && !lat->elec_on) return 0;
    int t, c[3];
    site_coords(lat, s, &t, c);
    int64_t E = lat->elec_on ? lat->elec_u[s] : 0;
    for (int i = 0; i < lat->n_vv; i++) {
        int64_t u = site_index(lat, lat->vv[t][i].t2, wrap(c[0] + lat->vv[t][i].dc[0], lat->L[0]),
                               wrap(c[1] + lat->vv[t][i].dc[1], lat->L[1]),
                               wrap(c[2] + lat->vv[t][i].dc[2], lat->L[2]));
        if (u != exclude && lat->occ[u] == SP_V) E += lat->vv[t][i].e;
    }
    for (int i = 0; i < lat->n_fe; i++) {
        int x = wrap(c[0] + lat->feo[t][i].dc[0], lat->L[0]);
        int y = wrap(c[1] + lat->feo[t][i].dc[1], lat->L[1]);
        int z = wrap(c[2] + lat->feo[t][i].dc[2], lat->L[2]);
        if (lat->fe[((int64_t)z * lat->L[1] + y) * lat->L[0] + x]) E += lat->feo[t][i].e;
    }
    return E;
}

/* ------------------------------------------------------------------ */
/* Grains (Sec. "Oxygen diffusion in mu-scale BaTiO3 model"): a Voronoi
 * tessellation of the cells, periodic in all three directions.  Seed g sits at
 * X_d = mulhi(y_d, 256 L_d) in units of 1/256 cell (y = the Philox block (g, 0,
 * 0, 0) under the key (seed, replica, GRAIN)); a cell, centre 256 c + 128,
 * belongs to the nearest seed (squared minimum-image distance, exact
 * integers; ties to the smaller g).  A cell is a boundary cell when a cell of
 * another grain lies within Chebyshev distance `width` of it; an O site
 * belongs to the cell it is attached to (site n + a/2 e_t to cell n).  A hop
 * whose start or end site is a boundary site has its barrier raised by
 * barrier_eV (0.2 eV in the paper: 0.9 eV in total through the boundary).  */
/* ------------------------------------------------------------------ */
int orc_set_grains(orc_lattice* lat, int n_grains, int width, double barrier_eV)
{
    if (n_grains <= 1) { lat->grains_on = 0; return 0; }
    if (n_grains > 4096 || width < 1 || !(barrier_eV >= 0.0) || !(barrier_eV <= 10.0)) return -1;
    for (int k = 0; k < 3; k++) if (lat->L[k] < 2 * width + 1) return -1;
    int64_t ncell = (int64_t)lat->L[0] * lat->L[1] * lat->L[2];
    int64_t* X = (int64_t*)malloc(sizeof(int64_t) * 3 * (size_t)n_grains);
    uint64_t key[2];
    key_for(lat->seed, lat->replica, PURPOSE_GRAIN, key);
    for (int g = 0; g < n_grains; g++) {
        uint64_t ctr[4] = {(uint64_t)g, 0, 0, 0}, y[4];
        orc_philox4x64(ctr, key, y);
        for (int d = 0; d < 3; d++) X[3 * g + d] = (int64_t)mulhi64(y[d], (uint64_t)256 * (uint64_t)lat->L[d]);
    }
    free(lat->grain);
    free(lat->gbound);
    lat->grain = (int32_t*)malloc(sizeof(int32_t) * (size_t)ncell);
    lat->gbound = (uint8_t*)calloc((size_t)ncell, 1);
    for (int64_t c = 0; c < ncell; c++) {
        int64_t cc[3] = {c % lat->L[0], (c / lat->L[0]) % lat->L[1], c / ((int64_t)lat->L[0] * lat->L[1])};
        int best = 0;
        int64_t bd = -1;
        for (int g = 0; g < n_grains; g++) {
            int64_t d2 = 0;
            for (int d = 0; d < 3; d++) {
                int64_t box = 256 * (int64_t)lat->L[d];
                int64_t dd = 256 * cc[d] + 128 - X[3 * g + d];
                if (dd < 0) dd = -dd;
                if (box - dd < dd) dd = box - dd;
                d2 += dd * dd;
            }
            if (bd < 0 || d2 < bd) { bd = d2; best = g; }
        }
        lat->grain[c] = best;
    }
    for (int64_t c = 0; c < ncell; c++) {
        int cx = (int)(c % lat->L[0]), cy = (int)((c / lat->L[0]) % lat->L[1]);
        int cz = (int)(c / ((int64_t)lat->L[0] * lat->L[1]));
        for (int dz = -width; dz <= width && !lat->gbound[c]; dz++)
            for (int dy = -width; dy <= width && !lat->gbound[c]; dy++)
                for (int dx = -width; dx <= width; dx++) {
                    int64_t o = ((int64_t)wrap(cz + dz, lat->L[2]) * lat->L[1] + wrap(cy + dy, lat->L[1])) *
                                    lat->L[0] + wrap(cx + dx, lat->L[0]);
                    if (lat->grain[o] != lat->grain[c]) { lat->gbound[c] = 1; break; }
                }
    }
    free(X);
    lat->gb_eV = barrier_eV;
    lat->grains_on = 1;
    if (lat->rates_set) {
        const double* a = lat->rate_args;
        return orc_set_rates(lat, a[0], a[1], a[2], a[3], a[4], a[5], a[6], a[7], lat->rate_cap, lat->rate_ntau,
                             lat->precision);
    }
    return 0;
}

void orc_get_grains(const orc_lattice* lat, int32_t* grain, uint8_t* boundary)
{
    int64_t ncell = (int64_t)lat->L[0] * lat->L[1] * lat->L[2];
    for (int64_t c = 0; c < ncell; c++) {
        grain[c] = lat->grains_on ? lat->grain[c] : 0;
        boundary[c] = lat->grains_on ? lat->gbound[c] : 0;
    }
}

/* 1 when the hop between sites s and j touches a boundary cell */
static int boundary_hop(const orc_lattice* lat, int64_t s, int64_t j)
{
    if (!lat->grains_on) return 0;
    int64_t ncell = (int64_t)lat->L[0] * lat->L[1] * lat->L[2];
    return lat->gbound[s % ncell] || lat->gbound[j % ncell];
}

/* rate of the event (vacancy at s of type t, ion at its neighbour n = j) of
 * table rate k0 */
static double site_rate(const orc_lattice* lat, int64_t s, int64_t j, int t, int n, double k0)
{
    int64_t m = orc_site_energy(lat, j, s) - orc_site_energy(lat, s, -1);
    if (lat->elec_on) m -= lat->elec_g[t][n];
    int64_t m1 = m >= 0 ? m / 512 : -((-m + 511) / 512);
    int64_t m0 = m - 512 * m1;
    double c = 1e-4 / (2.0 * (KB_EV * lat->T));
    double f1 = exp(-((double)(512 * m1) * c));
    double f0 = exp(-((double)m0 * c));
    double k = k0 * f1;
    return k * f0;
}

/* rate type of the event "vacancy at s exchanges with neighbour n", or -1 */
static int event_type(const orc_lattice* lat, int64_t s, int n)
{
    int t, c[3];
    site_coords(lat, s, &t, c);
    int64_t j = neighbour_site(lat, s, n);
    int sp = lat->occ[j];
    if (sp == SP_V) return -1;
    return 3 * sp + NB[t][n].d[2] + 1;
}

/* FP64 rate of the event (s, n): the table rate, times the site-energy
 * factor when the interactions are on; 0 when the neighbour is a vacancy */
static double event_rate64(const orc_lattice* lat, int64_t s, int n)
{
    int ty = event_type(lat, s, n);
    if (ty < 0) return 0.0;
    int64_t j = neighbour_site(lat, s, n);
    double k0 = boundary_hop(lat, s, j) ? lat->k64g[ty] : lat->k64[ty];
    if (!lat->site_on && !lat->elec_on) return k0;
    int t, c[3];
    site_coords(lat, s, &t, c);
    return site_rate(lat, s, j, t, n, k0);
}

/* fixed-point rate of the event (s, n) of the mixed form */
static uint64_t event_rate_q(const orc_lattice* lat, int64_t s, int n)
{
    int ty = event_type(lat, s, n);
    if (ty < 0) return 0;
    return boundary_hop(lat, s, neighbour_site(lat, s, n)) ? lat->qg[ty] : lat->q[ty];
}

double orc_event_rate(const orc_lattice* lat, int64_t s, int n) { return event_rate64(lat, s, n); }

static int cmp_rec(const void* a, const void* b)
{
    const orc_rec* p = (const orc_rec*)a;
    const orc_rec* q = (const orc_rec*)b;
    return p->site < q->site ? -1 : (p->site > q->site ? 1 : 0);
}

/* Inclusive prefix of the plain-form rates in the canonical order: chunks of
 * 32 events; inside a chunk a Kogge-Stone ladder (strides 1,2,4,8,16, each
 * element adding the element `stride` below it, all from the previous rung);
 * chunks joined by a running carry.  Returns the total.               */
static double canonical_prefix(const double* r, double* P, int nev)
{
    int nch = (nev + 31) / 32;
    double carry = 0.0;
    for (int c = 0; c < nch; c++) {
        double v[32];
        for (int l = 0; l < 32; l++) v[l] = (32 * c + l < nev) ? r[32 * c + l] : 0.0;
        for (int off = 1; off < 32; off *= 2)
            for (int l = 31; l >= off; l--) v[l] = v[l] + v[l - off];
        for (int l = 0; l < 32; l++)
            if (32 * c + l < nev) P[32 * c + l] = carry + v[l];
        carry = carry + v[31];
    }
    return carry;
}

/* One fragment F in window w: BKL on F's own vacancies until the next
 * event would pass the window length. */
static void fkmc_phase(orc_lattice* lat, int F, uint64_t w)
{
    orc_list* lst = &lat->frag[F];
    int n = lst->n;
    if (n == 0) return;
    orc_rec* slot = (orc_rec*)malloc(sizeof(orc_rec) * n);
    memcpy(slot, lst->r, sizeof(orc_rec) * n);
    qsort(slot, n, sizeof(orc_rec), cmp_rec); /* slots in ascending site order */
    int* alive = (int*)malloc(sizeof(int) * n);
    for (int m = 0; m < n; m++) alive[m] = 1;
    int nev = 8 * n;
    double* r64 = (double*)malloc(sizeof(double) * nev);
    double* P64 = (double*)malloc(sizeof(double) * nev);
    uint64_t* rq = (uint64_t*)malloc(sizeof(uint64_t) * nev);
    uint64_t key[2];
    key_for(lat->seed, lat->replica, PURPOSE_HOP, key);
    double clock = 0.0;
    uint64_t i = 0;
    uint64_t blk[4] = {0, 0, 0, 0};
    uint64_t blk_id = ~(uint64_t)0;
    for (;;) {
        /* rates of every event of F, Eq. (RateCnst1) table lookups (times
         * the site-energy factor when the interactions are on) */
        for (int m = 0; m < n; m++)
            for (int nb = 0; nb < 8; nb++) {
                int e = 8 * m + nb;
                int ty = alive[m] ? event_type(lat, slot[m].site, nb) : -1;
                r64[e] = ty < 0 ? 0.0 : event_rate64(lat, slot[m].site, nb);
                rq[e] = ty < 0 ? 0 : event_rate_q(lat, slot[m].site, nb);
            }
        /* draws of event i: Philox block (F, w, i/2); even i takes words 0,1 */
        if ((i >> 1) != blk_id) {
            uint64_t ctr[4] = {(uint64_t)F, w, i >> 1, 0};
            orc_philox4x64(ctr, key, blk);
            blk_id = i >> 1;
        }
        uint64_t xt = (i & 1) ? blk[2] : blk[0];
        uint64_t xs = (i & 1) ? blk[3] : blk[1];
        int e_sel = -1;
        double dclock;
        if (lat->precision == 0) {
            double R = canonical_prefix(r64, P64, nev);
            if (!(R > 0.0)) break;
            /* Eq. (TimeStep) */
            double dt = orc_neglog64(xt) / R;
            if (clock + dt > lat->tau) break;
            dclock = dt;
            /* Eq. (eventSelection): first event whose cumulative rate exceeds r*R */
            double target = (double)(xs >> 11) * 0x1p-53 * R;
            for (int e = 0; e < nev; e++)
                if (r64[e] > 0.0 && P64[e] > target) { e_sel = e; break; }
            if (e_sel < 0)
                for (int e = nev - 1; e >= 0; e--)
                    if (r64[e] > 0.0) { e_sel = e; break; }
        } else {
            uint64_t S = 0;
            for (int e = 0; e < nev; e++) S += rq[e];
            if (S == 0) break;
            /* clock in units of 1/k32max: dtheta = E * 2^F / S */
            float E = orc_neglog32(xt);
            float ratio = E / (float)S;
            double dth = ldexp((double)ratio, lat->F);
            if (clock + dth > lat->theta_tau) break;
            dclock = dth;
            uint64_t target = mulhi64(xs, S);
            uint64_t P = 0;
            for (int e = 0; e < nev; e++) {
                P += rq[e];
                if (P > target) { e_sel = e; break; }
            }
        }
        /* apply the exchange */
        int m = e_sel / 8, nb = e_sel % 8;
        int64_t s = slot[m].site;
        int t, c[3];
        site_coords(lat, s, &t, c);
        int64_t j = neighbour_site(lat, s, nb);
        int ion = lat->occ[j];
        lat->occ[s] = (uint8_t)ion;
        lat->occ[j] = SP_V;
        for (int k = 0; k < 3; k++) slot[m].d[k] += NB[t][nb].d[k];
        if (lat->tracer) {
            for (int k = 0; k < 3; k++) {
                lat->tdisp[3 * s + k] = lat->tdisp[3 * j + k] - NB[t][nb].d[k];
                lat->tdisp[3 * j + k] = 0;
            }
        }
        int G = fragment_of_site(lat, j);
        if (G == F) {
            slot[m].site = j;
        } else {
            orc_rec moved = slot[m];
            moved.site = j;
            list_push(&lat->frag[G], moved);
            alive[m] = 0;
            lat->handoffs++;
        }
        clock = clock + dclock;
        i++;
    }
    lat->hops += i;
    lat->clock_sum += clock;
    /* surviving records stay with F */
    lst->n = 0;
    for (int m = 0; m < n; m++)
        if (alive[m]) list_push(lst, slot[m]);
    free(slot); free(alive); free(r64); free(P64); free(rq);
}

int orc_run(orc_lattice* lat, uint64_t windows)
{
    if (!lat->rates_set) return -1;
    for (uint64_t k = 0; k < windows; k++) {
        uint64_t w = lat->window;
        int32_t perm[8];
        orc_colour_perm(lat->seed, lat->replica, w, perm);
        for (int p = 0; p < 8; p++)
            for (int F = 0; F < lat->nfrag; F++)
                if (fragment_colour(lat, F) == perm[p]) fkmc_phase(lat, F, w);
        lat->window++;
    }
    return 0;
}

/* ------------------------------------------------------------------ */
/* Conventional (non-fragmented) BKL of Sec. II.A on the same lattice, for
 * the statistical pins: all vacancies' events in one list, plain serial
 * cumulative sum, FP64 clock.  Runs until the clock passes t_end.      */
/* ------------------------------------------------------------------ */
int orc_bkl_run(orc_lattice* lat, double t_end, uint64_t stream, double* t_out)
{
    if (!lat->rates_set) return -1;
    int n = 0;
    for (int f = 0; f < lat->nfrag; f++) n += lat->frag[f].n;
    if (n == 0) { *t_out = t_end; return 0; }
    orc_rec* v = (orc_rec*)malloc(sizeof(orc_rec) * n);
    n = 0;
    for (int f = 0; f < lat->nfrag; f++)
        for (int k = 0; k < lat->frag[f].n; k++) v[n++] = lat->frag[f].r[k];
    qsort(v, n, sizeof(orc_rec), cmp_rec);
    double* r = (double*)malloc(sizeof(double) * 8 * n);
    uint64_t key[2];
    key_for(lat->seed, lat->replica, PURPOSE_BKL, key);
    double t = 0.0;
    uint64_t i = 0;
    for (;;) {
        double R = 0.0;
        for (int m = 0; m < n; m++)
            for (int nb = 0; nb < 8; nb++) {
                r[8 * m + nb] = event_rate64(lat, v[m].site, nb);
                R += r[8 * m + nb];
            }
        if (!(R > 0.0)) { t = t_end; break; }
        uint64_t ctr[4] = {stream, i, 0, 0}, y[4];
        orc_philox4x64(ctr, key, y);
        double dt = orc_neglog64(y[0]) / R;
        if (t + dt > t_end) { t = t_end; break; }
        double target = (double)(y[1] >> 11) * 0x1p-53 * R;
        double P = 0.0;
        int e_sel = -1, last = -1;
        for (int e = 0; e < 8 * n; e++) {
            if (r[e] > 0.0) last = e;
            P += r[e];
            if (r[e] > 0.0 && P > target) { e_sel = e; break; }
        }
        if (e_sel < 0) e_sel = last;
        int m = e_sel / 8, nb = e_sel % 8;
        int tt, c[3];
        site_coords(lat, v[m].site, &tt, c);
        int64_t j = neighbour_site(lat, v[m].site, nb);
        int ion = lat->occ[j];
        lat->occ[v[m].site] = (uint8_t)ion;
        lat->occ[j] = SP_V;
        for (int k = 0; k < 3; k++) v[m].d[k] += NB[tt][nb].d[k];
        if (lat->tracer)
            for (int k = 0; k < 3; k++) {
                lat->tdisp[3 * v[m].site + k] = lat->tdisp[3 * j + k] - NB[tt][nb].d[k];
                lat->tdisp[3 * j + k] = 0;
            }
        v[m].site = j;
        t = t + dt;
        i++;
    }
    /* records back to their owning fragments */
    for (int f = 0; f < lat->nfrag; f++) lat->frag[f].n = 0;
    for (int m = 0; m < n; m++) list_push(&lat->frag[fragment_of_site(lat, v[m].site)], v[m]);
    lat->hops += i;
    *t_out = t;
    free(v); free(r);
    return 0;
}

/* ------------------------------------------------------------------ */
/* The atom-based fragment kMC of Sec. II.B with null events, the atoms I
 * being the vacancies (each with its 8 exchanges).  One step:
 *  1. R_I = the sum of vacancy I's rates, R_tot = sum_I R_I and
 *     R_max = max_I R_I (Eq. AtomP).  Rates are the mixed form's fixed point
 *     with F_null = 63 - ceil(log2(8 N_V)), so every sum is an exact integer
 *     below 2^63.
 *  2. N_frg distinct vacancies are picked: the images of 0 .. N_frg-1 under
 *     a keyed bijection of the vacancy ids (an alternating Feistel network
 *     with per-step round keys, null_pick below).  The paper says only that
 *     the atoms are selected at random.
 *  3. Pick p draws x and takes the first of its vacancy's events whose
 *     running sum exceeds mulhi(x, R_max) -- probability k_i / R_max -- or the
 *     null event when R_I does not (probability 1 - R_I / R_max).
 *  4. The paper leaves open how simultaneous picks are reconciled.  Reading:
 *     a pick whose exchange shares a site with the exchange of a non-null
 *     pick of smaller index becomes null, so the updated events are disjoint
 *     and commute.
 *  5. The exchanges are applied; N_updated is their number and the clock
 *     moves by -ln(r') / R_tot * N_updated (Eq. TimeStepFrg).
 * With N_frg = 1 this is the conventional kMC of Sec. II.A in distribution.
 */
/* ------------------------------------------------------------------ */
int64_t orc_n_records(const orc_lattice* lat);

/* 64-bit finaliser of MurmurHash3 (Appleby): xor-shift 33, multiply, xor-shift
 * 33, multiply, xor-shift 33, with its two published odd multipliers. */
static uint64_t fmix64(uint64_t h)
{
    h ^= h >> 33;
    h *= 0xff51afd7ed558ccdull;
    h ^= h >> 33;
    h *= 0xc4ceb9fe1a85ec53ull;
    h ^= h >> 33;
    return h;
}

/* Pick p of step `step`: the image of p under a keyed bijection of [0, n):
 * an alternating Feistel network on m = max(2, ceil(log2 n)) bits (high part
 * m - m/2 bits, low part m/2 bits; round r = 0..11 XORs F_r of one part into
 * the other, high first), with cycle walking (Black & Rogaway) back into
 * [0, n).  F_r(x) = fmix64(x ^ k_r); the round keys k_0..k_11 are the Philox
 * blocks (step, j, 0, 0), j = 0, 1, 2, under the key (seed, replica, PICK),
 * k_{4j+i} = word i of block j.  Twelve rounds make the permutation of a
 * small domain (n = 3..6) close to uniform over all n! orders; four are not. */
#define NULL_PICK_ROUNDS 12
static uint64_t null_pick(uint64_t p, uint64_t n, uint64_t seed, uint32_t replica, uint64_t step)
{
    int m = 2;
    while (((uint64_t)1 << m) < n) m++;
    int bl = m / 2, bh = m - bl;
    uint64_t ml = ((uint64_t)1 << bl) - 1, mh = ((uint64_t)1 << bh) - 1;
    uint64_t key[2], k[NULL_PICK_ROUNDS];
    key_for(seed, replica, PURPOSE_PICK, key);
    for (int j = 0; j < NULL_PICK_ROUNDS / 4; j++) {
        uint64_t ctr[4] = {step, (uint64_t)j, 0, 0};
        orc_philox4x64(ctr, key, k + 4 * j);
    }
    uint64_t v = p;
    do {
        uint64_t hi = v >> bl, lo = v & ml;
        for (int r = 0; r < NULL_PICK_ROUNDS; r++) {
            if (r % 2 == 0) hi = hi ^ (fmix64(lo ^ k[r]) & mh);
            else lo = lo ^ (fmix64(hi ^ k[r]) & ml);
        }
        v = (hi << bl) | lo;
    } while (v >= n);
    return v;
}

uint64_t orc_null_pick(uint64_t p, uint64_t n, uint64_t seed, uint32_t replica, uint64_t step)
{
    return null_pick(p, n, seed, replica, step);
}

/* fixed-point tables of the null-event form for N_V vacancies: q[0..5] bulk
 * hops, q[6..11] boundary hops (grains) */
static int null_table(const orc_lattice* lat, int64_t nv, uint64_t q[12])
{
    float kmax = 0.0f;
    for (int i = 0; i < 6; i++) if (lat->k32[i] > kmax) kmax = lat->k32[i];
    int lg = 0;
    while (((int64_t)1 << lg) < 8 * (nv > 0 ? nv : 1)) lg++;
    int F = 63 - lg;
    for (int i = 0; i < 6; i++) q[i] = (uint64_t)llrint(ldexp((double)lat->k32[i] / (double)kmax, F));
    for (int i = 0; i < 6; i++)
        q[6 + i] = lat->grains_on ? (uint64_t)llrint(ldexp((double)lat->k32g[i] / (double)kmax, F)) : q[i];
    return F;
}

static uint64_t null_q(const orc_lattice* lat, const uint64_t q[12], int64_t s, int n)
{
    int ty = event_type(lat, s, n);
    if (ty < 0) return 0;
    return q[ty + (boundary_hop(lat, s, neighbour_site(lat, s, n)) ? 6 : 0)];
}

int orc_null_run(orc_lattice* lat, uint64_t steps, int64_t n_frg)
{
    if (!lat->rates_set || lat->site_on || lat->elec_on || n_frg < 1) return -1;
    int64_t nv = orc_n_records(lat);
    if (nv == 0) { lat->null_step += steps; return 0; }
    orc_rec* v = (orc_rec*)malloc(sizeof(orc_rec) * nv);
    for (int f = 0; f < lat->nfrag; f++)
        for (int m = 0; m < lat->frag[f].n; m++) {
            orc_rec r = lat->frag[f].r[m];
            if ((int64_t)r.id >= nv) { free(v); return -1; }
            v[r.id] = r; /* vacancy ids are 0 .. N_V-1 */
        }
    if (!lat->claimed) lat->claimed = (int64_t*)calloc((size_t)lat->nsite, sizeof(int64_t));
    uint64_t q[12];
    int F = null_table(lat, nv, q);
    int64_t nf = n_frg < nv ? n_frg : nv;
    uint64_t key[2];
    key_for(lat->seed, lat->replica, PURPOSE_NULL, key);
    int64_t* pv = (int64_t*)malloc(sizeof(int64_t) * nf);
    int* pn = (int*)malloc(sizeof(int) * nf);
    for (uint64_t k = 0; k < steps; k++) {
        uint64_t step = lat->null_step;
        /* 1. per-vacancy totals */
        uint64_t Rtot = 0, Rmax = 0;
        for (int64_t i = 0; i < nv; i++) {
            uint64_t R = 0;
            for (int n = 0; n < 8; n++) R += null_q(lat, q, v[i].site, n);
            Rtot += R;
            if (R > Rmax) Rmax = R;
        }
        /* 2-3. picks and their proposals, all from the state before the step */
        for (int64_t p = 0; p < nf; p++) {
            int64_t id = (int64_t)null_pick((uint64_t)p, (uint64_t)nv, lat->seed, lat->replica, step);
            uint64_t ctr[4] = {step, (uint64_t)p, 0, 0}, y[4];
            orc_philox4x64(ctr, key, y);
            uint64_t target = mulhi64(y[0], Rmax);
            uint64_t P = 0;
            int sel = -1;
            for (int n = 0; n < 8; n++) {
                P += null_q(lat, q, v[id].site, n);
                if (P > target) { sel = n; break; }
            }
            pv[p] = id;
            pn[p] = sel;
        }
        /* 4. a non-null pick loses to any earlier non-null pick sharing a site */
        for (int64_t p = 0; p < nf; p++) {
            if (pn[p] < 0) continue;
            int64_t s = v[pv[p]].site, j = neighbour_site(lat, s, pn[p]);
            int clash = lat->claimed[s] == (int64_t)step + 1 || lat->claimed[j] == (int64_t)step + 1;
            lat->claimed[s] = lat->claimed[j] = (int64_t)step + 1;
            if (clash) pn[p] = -1;
        }
        /* 5. apply (disjoint, so in any order) and advance the clock */
        uint64_t nupd = 0;
        for (int64_t p = 0; p < nf; p++) {
            if (pn[p] < 0) continue;
            orc_rec* r = &v[pv[p]];
            int t, c[3];
            site_coords(lat, r->site, &t, c);
            int64_t s = r->site, j = neighbour_site(lat, s, pn[p]);
            int ion = lat->occ[j];
            lat->occ[s] = (uint8_t)ion;
            lat->occ[j] = SP_V;
            for (int d = 0; d < 3; d++) r->d[d] += NB[t][pn[p]].d[d];
            if (lat->tracer)
                for (int d = 0; d < 3; d++) {
                    lat->tdisp[3 * s + d] = lat->tdisp[3 * j + d] - NB[t][pn[p]].d[d];
                    lat->tdisp[3 * j + d] = 0;
                }
            r->site = j;
            nupd++;
        }
        if (Rtot > 0) {
            uint64_t ct[4] = {step, ~(uint64_t)0, 0, 0}, y[4];
            orc_philox4x64(ct, key, y);
            double E = orc_neglog64(y[0]);
            double dth = ldexp(E / (double)Rtot, F) * (double)nupd;
            lat->theta_null = lat->theta_null + dth;
        }
        lat->hops += nupd;
        lat->null_step++;
    }
    /* records back to the fragments owning their sites */
    for (int f = 0; f < lat->nfrag; f++) lat->frag[f].n = 0;
    for (int64_t i = 0; i < nv; i++) list_push(&lat->frag[fragment_of_site(lat, v[i].site)], v[i]);
    free(v); free(pv); free(pn);
    return 0;
}

/* clock of the null-event form: {theta (1/k32max units), t (s)}, steps and F_null */
void orc_get_null(const orc_lattice* lat, double* theta, double* t_s, uint64_t* steps, int32_t* F)
{
    uint64_t q[12];
    float kmax = 0.0f;
    for (int i = 0; i < 6; i++) if (lat->k32[i] > kmax) kmax = lat->k32[i];
    *theta = lat->theta_null;
    *t_s = kmax > 0.0f ? lat->theta_null / (double)kmax : 0.0;
    *steps = lat->null_step;
    *F = null_table(lat, orc_n_records(lat), q);
}

/* ------------------------------------------------------------------ */
/* Read-out                                                            */
/* ------------------------------------------------------------------ */
void orc_get_occ(const orc_lattice* lat, uint8_t* out) { memcpy(out, lat->occ, (size_t)lat->nsite); }

void orc_set_occ_records(orc_lattice* lat, const uint8_t* occ)
{
    /* replace the state: occupancy as given, one zero-displacement record per
     * vacancy with id = rank in site order; tracer displacements cleared */
    memcpy(lat->occ, occ, (size_t)lat->nsite);
    for (int f = 0; f < lat->nfrag; f++) lat->frag[f].n = 0;
    uint32_t id = 0;
    for (int64_t s = 0; s < lat->nsite; s++)
        if (occ[s] == SP_V) {
            orc_rec r = {s, {0, 0, 0}, id++};
            list_push(&lat->frag[fragment_of_site(lat, s)], r);
        }
    if (lat->tracer) memset(lat->tdisp, 0, sizeof(int32_t) * 3 * (size_t)lat->nsite);
}

int64_t orc_n_records(const orc_lattice* lat)
{
    int64_t n = 0;
    for (int f = 0; f < lat->nfrag; f++) n += lat->frag[f].n;
    return n;
}

/* records as rows {fragment, site, dx, dy, dz, id}, fragments ascending,
 * sites ascending inside a fragment */
int64_t orc_get_records(const orc_lattice* lat, int64_t* out, int64_t max_rows)
{
    int64_t k = 0;
    for (int f = 0; f < lat->nfrag; f++) {
        orc_list* l = &lat->frag[f];
        orc_rec* tmp = (orc_rec*)malloc(sizeof(orc_rec) * (l->n ? l->n : 1));
        memcpy(tmp, l->r, sizeof(orc_rec) * l->n);
        qsort(tmp, l->n, sizeof(orc_rec), cmp_rec);
        for (int m = 0; m < l->n && k < max_rows; m++, k++) {
            int64_t* o = out + 6 * k;
            o[0] = f; o[1] = tmp[m].site;
            o[2] = tmp[m].d[0]; o[3] = tmp[m].d[1]; o[4] = tmp[m].d[2]; o[5] = tmp[m].id;
        }
        free(tmp);
    }
    return k;
}

void orc_get_tracer(const orc_lattice* lat, int32_t* out)
{
    if (lat->tracer) memcpy(out, lat->tdisp, sizeof(int32_t) * 3 * (size_t)lat->nsite);
}

/* counters: {window, hops, handoffs} and the diagnostic clock sum */
void orc_get_counters(const orc_lattice* lat, uint64_t* out3, double* clock_sum)
{
    out3[0] = lat->window; out3[1] = lat->hops; out3[2] = lat->handoffs;
    *clock_sum = lat->clock_sum;
}

void orc_get_params(const orc_lattice* lat, double* tau, double* theta_tau, int32_t* F)
{
    *tau = lat->tau; *theta_tau = lat->theta_tau; *F = lat->F;
}

/* Second moments of the displacements (units (a/2)^2), exact integers:
 * species SP_V over vacancy records, SP_O / SP_H over the tracer field.
 * out: {count, sum dx, sum dy, sum dz, sum dx^2, sum dy^2, sum dz^2}    */
int orc_moments(const orc_lattice* lat, int species, int64_t* out)
{
    memset(out, 0, 7 * sizeof(int64_t));
    if (species == SP_V) {
        for (int f = 0; f < lat->nfrag; f++)
            for (int m = 0; m < lat->frag[f].n; m++) {
                const int32_t* d = lat->frag[f].r[m].d;
                out[0]++;
                for (int k = 0; k < 3; k++) { out[1 + k] += d[k]; out[4 + k] += (int64_t)d[k] * d[k]; }
            }
        return 0;
    }
    if (!lat->tracer) return -1;
    for (int64_t s = 0; s < lat->nsite; s++)
        if (lat->occ[s] == species) {
            const int32_t* d = lat->tdisp + 3 * s;
            out[0]++;
            for (int k = 0; k < 3; k++) { out[1 + k] += d[k]; out[4 + k] += (int64_t)d[k] * d[k]; }
        }
    return 0;
}
