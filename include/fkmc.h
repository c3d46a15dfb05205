/*
 * fkmc.h -- C ABI of the GB300 fragment kinetic Monte Carlo library.
 *
 * Method: H. Nakata, "Development of a fragment kinetic Monte Carlo method for
 * efficient prediction of ionic diffusion in perovskite crystals",
 * arXiv:2004.09081.  O vacancies (V) and hydride ions (H-) hop on the O
 * sublattice of a cubic ABO3 perovskite (Fig. 2: O at the three face centres
 * of a cell of edge a, 8 O-O neighbours at a/sqrt2).  Hop rates follow
 * Eq. (RateCnst1), k = A exp(-Ea/(kB T)), with the electrostatic shift of
 * Sec. III; events are selected by cumulative rate, Eq. (eventSelection), and
 * each fragment keeps its own residence-time clock, Eq. (TimeStep).  Fragments
 * select independently because, once the clock is shared, an event's
 * probability depends only on the rates it competes with (Sec. II.B,
 * Eq. (AtomP)).
 *
 * Execution model: the lattice is cut into spatial fragments (an even number
 * per dimension, or one); fragments are coloured by the parity of their
 * indices (8 colours).  A synchronisation window of length tau runs the 8
 * colours in a per-window random order; in a colour phase every fragment of
 * that colour runs BKL on its own vacancies until its next event would pass
 * tau.  Concurrent fragments never touch the same site.  A vacancy that hops
 * out of its fragment is handed to the owner of its new site and moves again
 * when that fragment's colour next runs.  Global time after window w is
 * (w+1) tau.
 *
 * Conventions for every entry point:
 *   - Return value: FKMC_OK (0) or a negative FKMC_E* code; kmc_last_error()
 *     returns a thread-local message for the last failure.  Nothing aborts.
 *   - Host pointers are read or written only during the call; the library
 *     keeps no reference to them.  Device memory belongs to the batch (taken
 *     from the caller's allocator callback if given, else cudaMalloc) and is
 *     released by kmc_destroy().
 *   - All GPU work goes to the stream in kmc_opts.stream (NULL = legacy
 *     default stream).  kmc_run() and the read/write calls are synchronous on
 *     return.
 *   - Units: temperatures K, energies eV, fields V/m, lengths Angstrom in
 *     inputs; D in m^2/s, time in s in outputs.  Displacements are integers
 *     in units of a/2.
 */
#ifndef FKMC_ABI_H_
#define FKMC_ABI_H_

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define FKMC_OK 0
#define FKMC_EINVAL (-1)    /* bad argument: sizes, partition, composition, replica index */
#define FKMC_ENOMEM (-2)    /* allocator returned NULL */
#define FKMC_ECUDA (-3)     /* a CUDA runtime call failed (message has the CUDA error) */
#define FKMC_ETIMEOUT (-4)  /* a device-side wait or the per-phase event bound (2^24) ran out */
#define FKMC_EOVERFLOW (-5) /* a fragment received more vacancies than its slot capacity */
#define FKMC_ESTATE (-6)    /* call out of order (e.g. kmc_run before kmc_set_barriers) */

/* species codes (2 bits per site on the device) */
#define FKMC_O 0
#define FKMC_H 1
#define FKMC_V 2

/* arithmetic forms */
#define FKMC_PLAIN 0 /* FP64 rates, FP64 prefix sums, FP64 clock */
#define FKMC_MIXED 1 /* FP32 rates quantised to u64 fixed point, exact integer sums, FP32 variate + FP64 clock */

typedef struct {
    int32_t nx, ny, nz; /* cells per dimension, each >= 1 and <= 65535 */
    double a_angstrom;  /* cubic lattice constant */
} kmc_cells;

typedef struct {
    int64_t n_vac; /* O vacancies placed at creation */
    int64_t n_H;   /* H- ions placed at creation (on O sites) */
    int64_t n_Fe;  /* dopants placed at creation on the B sites (cell corners); they do not move and
                      act only through the site energies of kmc_set_site_energy */
} kmc_composition;

/* Site-energy interactions (the dopant/defect section of the paper and its
 * Table add01): the energy of a vacancy at O site s is
 *   E_site(s) = sum_k N_VV,k(s) vv_eV[k] + sum_k N_VFe,k(s) fe_eV[k],
 * N counting the other vacancies at squared O-O distance vv_d2[k] and the
 * dopants at squared O-B distance fe_d2[k] from s (both in units of (a/2)^2:
 * O-O shells are even, 2 = a/sqrt2, 4 = a, 6, 8, 10, ...; O-B shells odd,
 * 1 = a/2, 5, 9, 13, ...).  The hop s -> j then has barrier
 * Ea + dU/2 + (E_site(j) - E_site(s))/2, E_site(j) counted without the hopping
 * vacancy (the energy change of the whole configuration, so detailed balance
 * holds).  Energies are rounded to multiples of 1e-4 eV (rint(e * 1e4)); the
 * factor exp(-dE/(2 kB T)) of an energy difference of m such units is
 * exp(-(512 m1) c) * exp(-m0 c), m = 512 m1 + m0, 0 <= m0 < 512,
 * c = 1e-4 / (2 kB T), multiplied into the table rate in that order. */
#define FKMC_MAX_SHELLS 8
typedef struct {
    int32_t n_vv;                   /* V-V shells in use, 0..8 */
    int32_t vv_d2[FKMC_MAX_SHELLS]; /* squared O-O distance of each shell, (a/2)^2 units */
    double vv_eV[FKMC_MAX_SHELLS];  /* pair energy of a vacancy in that shell, eV */
    int32_t n_fe;                   /* vacancy-dopant shells in use, 0..8 */
    int32_t fe_d2[FKMC_MAX_SHELLS]; /* squared O-B distance of each shell, (a/2)^2 units */
    double fe_eV[FKMC_MAX_SHELLS];  /* pair energy of a vacancy and a dopant in that shell, eV */
} kmc_site_energy;

typedef struct {
    double Ea_O_eV;   /* barrier of the O <-> V exchange */
    double Ea_H_eV;   /* barrier of the H- <-> V exchange */
    double prefactor; /* A of Eq. (RateCnst1), 1/s (the paper uses 1e13) */
    double q_O;       /* charge carried with the vacancy in an O exchange, units of e (+2) */
    double q_H;       /* same for an H- exchange (+1) */
} kmc_barrier_table;

typedef void* (*kmc_alloc_fn)(void* ctx, size_t bytes);
typedef void (*kmc_free_fn)(void* ctx, void* ptr);

typedef struct {
    int32_t edge;       /* target fragment edge in cells (used where nfrag[d] == 0); default 4 */
    int32_t nfrag[3];   /* fragments per dimension: 1 or even with every edge >= 2; 0 = from edge */
    int32_t precision;  /* FKMC_PLAIN or FKMC_MIXED */
    int32_t tracer;     /* nonzero: also track every ion's displacement (12 bytes per site) */
    int32_t cap_v;      /* vacancy slots per fragment, 8..256; 0 = sized from the composition */
    double n_tau;       /* window length tau = n_tau / (8 k_fast), 0 < n_tau <= 64; default 1 */
    void* stream;       /* cudaStream_t for all work */
    kmc_alloc_fn alloc; /* optional device allocator; NULL = cudaMalloc */
    kmc_free_fn free;
    void* alloc_ctx;
    int32_t schedule;   /* 0 = auto: mixed-form replicas whose state fits one SM run in the
                           replica-resident kernel, the rest one launch per colour phase;
                           1 = colour-phase launches only; 2 = resident kernel only */
    int32_t cluster_top; /* resident kernel: how many of the largest replicas of the 1024-thread
                            class run as 2-CTA thread-block clusters (each CTA holds the replica
                            and takes half of every phase's fragments; writes are mirrored
                            through distributed shared memory).  -1 (default) = SMs / 8,
                            0 = none */
    int32_t small_pass; /* colour-phase kernels: sparse fragments run in a pass of their own besides
                           the general one (one warp per fragment); same trajectory.  Mixed form:
                           one thread per fragment (see lane_form); plain form (and mode 2):
                           fragments holding one or two vacancies, 4 or 2 per warp in lock-step.
                           0 (default) = where a phase holds 32768 fragments or more,
                           1 = always, 2 = always and in the grouped form, -1 = never */
    int32_t test_stuck_wait_us; /* test of the device-side bounded wait (0 = off): the replica-resident
                                   kernel, after staging its state, waits on a barrier that nothing
                                   completes, gives up after this many microseconds (<= 2e6) and
                                   kmc_run returns FKMC_ETIMEOUT with the state untouched */
    int32_t lane_form;  /* mixed form, one-thread-per-fragment pass: 0 (default) = by phase size,
                           1 = registers (up to 4 vacancies, beside the general pass),
                           2 = persistent (up to 8 vacancies in shared memory, a grid that
                           stays resident for the phase; the general pass after it) */
    int32_t cluster_ctas; /* mixed form: a replica too large for one SM's shared memory runs in the
                             cluster-resident kernel (a thread-block cluster of up to 16 CTAs,
                             each holding a z-slab of fragment layers in shared memory, peers'
                             slabs reached through distributed shared memory) where its slabs
                             fit.  0 (default) = so, with the fewest CTAs that fit; -1 = never
                             (the colour-phase kernels); 2..16 = every replica with that many
                             fragment layers or more, with exactly this many CTAs */
    int32_t reserved[2];
} kmc_opts;

typedef struct {
    uint64_t hops;     /* executed (non-null) exchanges, summed over replicas */
    uint64_t handoffs; /* exchanges that moved a vacancy into another fragment */
    uint64_t windows;  /* windows run by this call */
    double gpu_ms;     /* device time of the call's kernels (CUDA events) */
    uint64_t launches; /* kernel launches made by the call */
} kmc_run_stats;

typedef struct {
    int32_t nfrag[3];   /* fragments per dimension */
    int32_t cap_v;      /* vacancy slots per fragment */
    int32_t F;          /* fixed-point fraction bits of the mixed form */
    int32_t precision;
    double tau;         /* window length, s */
    double theta_tau;   /* window length in units of 1/k32max (mixed clock) */
    double k64[6];      /* FP64 rate table, index 3*h + dz + 1 (h: 0 = O, 1 = H) */
    uint64_t q[6];      /* fixed-point table of the mixed form */
    uint64_t window;    /* windows completed */
    uint64_t hops;      /* exchanges executed so far */
    uint64_t handoffs;
    int64_t nsite;      /* 3 nx ny nz */
    int64_t n_vac, n_H;
    uint64_t null_steps; /* steps of the null-event form run so far (kmc_run_null) */
    double null_theta;   /* its clock in units of 1/k32max */
    double null_time_s;  /* its simulated time, s (included in kmc_read_msd's t) */
    int64_t n_Fe;        /* dopants */
    int32_t kernel;      /* how kmc_run advances the replica under the current rates and options:
                            0 = colour-phase kernels (one launch per phase), 1 = replica-resident
                            kernel (state in one SM's shared memory, or a 2-CTA mirrored pair),
                            2 = cluster-resident kernel (z-slabs in a thread-block cluster) */
    int32_t ctas;        /* CTAs holding the replica (kernels 1 and 2), else 0 */
    int32_t draw_phases; /* kernel 1: colour phases whose fragments' first random draws the kernel
                            makes in one batch (8, 4, 2 or 1, as the replica's shared-memory class
                            leaves room), else 0 */
    int32_t draw_events; /* kernel 1: events per fragment and phase drawn in that batch (4 where
                            2 or more phases of them fit, else 2), else 0 */
} kmc_replica_info;

typedef struct kmc_batch kmc_batch;

/* Fill *opts with the defaults listed above. */
void kmc_default_opts(kmc_opts* opts);

/* Create n independent replicas (lattices of possibly different sizes and
 * compositions) in one batch; replica r uses cells[r], comp[r] and draws its
 * random numbers from Philox4x64-10 keyed by (seed, r).  The initial state
 * places comp[r].n_vac vacancies and then comp[r].n_H hydride ions at the
 * images of 0, 1, 2, ... under a keyed bijection of the site indices (a
 * 4-round Feistel network with cycle walking); vacancy i gets id i.  The
 * paper gives no placement rule; this one gives exact counts and uniformly
 * random positions.  Dopants take the cells at the images of 0 ..
 * comp[r].n_Fe - 1 under the same construction over the cell indices with
 * its own key.
 * Errors: FKMC_EINVAL for n < 1, bad cells/partition/composition or opts;
 * FKMC_ENOMEM / FKMC_ECUDA; FKMC_EOVERFLOW if a fragment starts with more
 * vacancies than cap_v.  On error *out is NULL and nothing is leaked. */
int kmc_create_batch(int32_t n, const kmc_cells* cells, const kmc_composition* comp,
                     uint64_t seed, const kmc_opts* opts, kmc_batch** out);

/* kmc_create_batch with n = 1. */
int kmc_create_lattice(const kmc_cells* cells, const kmc_composition* comp, uint64_t seed,
                       const kmc_opts* opts, kmc_batch** out);

/* Rate tables of every replica, Eq. (RateCnst1) with the ESP shift of Sec. III:
 *   k[h][dz] = A exp(-(Ea_h + dU/2) / (kB T)),  dU = -q_h E_z dz a/2,
 * dz in {-1,0,+1} the vacancy's z step in units of a/2 (in-plane hops have
 * dz = 0).  tables, T_K and field_z_Vpm each hold n entries (field may be
 * NULL = 0).  Computed on the host in FP64; the mixed form stores
 * k32 = fp32(k64) and q = rint(k32/k32max 2^F), F = 63 - ceil(log2(8 cap_v)).
 * Sets tau = n_tau / (8 k_fast), k_fast the largest rate of the species
 * present.  Errors: FKMC_EINVAL for T <= 0 or non-finite inputs. */
int kmc_set_barriers(kmc_batch* b, const kmc_barrier_table* tables, const double* T_K,
                     const double* field_z_Vpm);

/* Turn the site-energy interactions on for every replica of the batch (e
 * NULL, or no shells, turns them off).  Plain form only: the event rates are
 * FP64 products of the table rate and the Boltzmann factor above, summed in
 * the canonical order.  Every replica then runs the colour-phase kernels
 * (the replica-resident kernel has no site energies).  The library keeps an
 * int32 energy field of every O site (4 bytes per site), rebuilt from the
 * vacancies and dopants at the next kmc_run after any state change, and
 * moved with each hop.
 * Errors: FKMC_EINVAL for the mixed form, more than 8 shells, a squared
 * distance that is not a shell of the lattice or above 36, |energy| > 10 eV,
 * a dimension shorter than 2 R + 1 cells (R = the largest cell offset of any
 * shell: a partner would be counted twice) or, where a dimension has more
 * than one fragment, a fragment edge below 2 + R_VV (R_VV from the V-V
 * shells: same-colour fragments would then read each other's writes);
 * FKMC_ENOMEM; FKMC_ECUDA. */
int kmc_set_site_energy(kmc_batch* b, const kmc_site_energy* e);

/* Host-only: the partner table of e for an O site of type t: rows
 * {t2, dcx, dcy, dcz, energy} of the V-V partners (O site type t2 in the cell
 * offset dc) followed by rows {-1, dcx, dcy, dcz, energy} of the B sites in
 * the dopant shells; energies in 1e-4 eV units.  *n_rows gets the row count,
 * at most max_rows rows are written.  Errors as kmc_set_site_energy's shell
 * checks. */
int kmc_site_shells(const kmc_site_energy* e, int32_t t, int32_t* rows, int32_t max_rows, int32_t* n_rows);

/* Dopants of replica r, one byte per cell (1 = doped), cell index
 * (z ny + y) nx + x.  kmc_write_dopants replaces them (the energy field is
 * rebuilt at the next kmc_run).  n must equal nx ny nz. */
int kmc_read_dopants(kmc_batch* b, int32_t r, uint8_t* host_cells, size_t n);
int kmc_write_dopants(kmc_batch* b, int32_t r, const uint8_t* host_cells, size_t n);

/* Energy field of replica r: E_site of every O site in 1e-4 eV units, site
 * index as in kmc_read_state (FKMC_ESTATE while the interactions are off). */
int kmc_read_site_field(kmc_batch* b, int32_t r, int32_t* host_field, size_t n);

/* Electrostatics (the mu-scale model section of the paper solves a Poisson
 * equation for the electrostatic potential).  Reading: the source is the
 * vacancies' own charge q_vac e, each split in halves between the two B sites
 * (cell corners) of its O site's bond, against a uniform neutralising
 * background, on the periodic grid of B sites (spacing a):
 *   6 phi(n) - sum_{6 neighbours} phi(n') = Q(n) / (eps0 eps_r a)      [V],
 * solved by a geometric multigrid (`cycles` V-cycles, red-black Gauss-Seidel,
 * full weighting, trilinear prolongation; deterministic).  The bias of the
 * paper stays the uniform field of kmc_set_barriers.  A vacancy at O site s
 * (the mean potential of its two nodes, phi(s)) has the energy
 * u(s) = rint(q_vac phi(s) 1e4) in 1e-4 eV units, added to the site energy of
 * kmc_set_site_energy; a hop s -> j of a type-t site to its neighbour n also
 * leaves out the vacancy's own potential, g[t][n] = rint(q_vac^2 (G(j, s) -
 * G(s, s)) 1e4), G the potential of a unit charge's deposit (one table per
 * replica, from three unit-charge solves).  The field is frozen between
 * refreshes: every `refresh_windows` windows kmc_run solves again from the
 * current vacancies (0: never; u stays as last solved or written).
 * Plain form only; the site-energy run pass of the colour-phase kernels. */
typedef struct {
    double eps_r;             /* relative permittivity, > 0 */
    double q_vac;             /* vacancy charge in e (+2 for an O vacancy) */
    int32_t refresh_windows;  /* windows between solves; 0 = no automatic solve */
    int32_t cycles;           /* V-cycles per solve, 1..200 (12 reach a relative residual ~1e-10) */
    int32_t warm_cycles;      /* V-cycles of an automatic refresh, which starts from the last
                                 solve's potential, 0..200 (0: `cycles`); the first solve after
                                 kmc_set_electrostatics or a state write starts from zero */
} kmc_electrostatics;

/* Turn electrostatics on (or off with NULL) for every replica and solve once.
 * Extra device memory: 4 bytes per O site, about 3 doubles per cell for the
 * multigrid levels of the largest replica.  Errors: FKMC_EINVAL for the mixed
 * form, bad parameters or a replica of 2^31 cells or more; FKMC_ENOMEM;
 * FKMC_ECUDA. */
int kmc_set_electrostatics(kmc_batch* b, const kmc_electrostatics* e);

/* Solve the potential of replica r's current vacancies (kmc_set_electrostatics
 * gives the parameters) without touching the state: phi at every B node (V),
 * index (z ny + y) nx + x, n = nx ny nz, and the relative residual
 * max|f - A phi| / max|f| (may be NULL).  FKMC_ESTATE without electrostatics. */
int kmc_solve_potential(kmc_batch* b, int32_t r, double* phi, size_t n, double* resid_rel);

/* The electrostatic energies u (int32 per O site, site index as in
 * kmc_read_state) of replica r and its own-potential table g (24 int32,
 * [t][n]; g may be NULL): read them, or write them (the caller's own potential;
 * set refresh_windows to 0 to keep them). */
int kmc_read_potential_energy(kmc_batch* b, int32_t r, int32_t* u, size_t n, int32_t* g);
int kmc_write_potential_energy(kmc_batch* b, int32_t r, const int32_t* u, size_t n, const int32_t* g);

/* Grains (the mu-scale model section of the paper): a periodic Voronoi
 * tessellation of each replica's cells.  Seed g of replica r sits at
 * X_d = mulhi(y_d, 256 L_d) in units of 1/256 cell, y the Philox4x64-10 block
 * (g, 0, 0, 0) under the key (seed, r << 8 | 8); a cell (centre 256 c + 128)
 * belongs to the nearest seed by squared minimum-image distance (exact
 * integers; ties to the smaller g).  A cell is a boundary cell when a cell of
 * another grain lies within Chebyshev distance `width`; an O site belongs to
 * the cell it is attached to (site n + a/2 e_t to cell n).  Every hop that
 * starts or ends on a boundary site has its barrier raised by barrier_eV (the
 * paper's 0.2 eV, 0.9 eV in total through a boundary): the mixed form
 * quantises those rates against the bulk table's k32max, so tau and F are
 * unchanged. */
typedef struct {
    int32_t n_grains;  /* seeds per replica, 2..4096; <= 1 turns grains off */
    int32_t width;     /* boundary-layer reach in cells, >= 1 (each dimension must be >= 2 width + 1) */
    double barrier_eV; /* added to the barrier of boundary hops, 0 .. 10 eV */
} kmc_grains;

/* Set (or with NULL / n_grains <= 1 clear) the grains of every replica.  The
 * grain map costs O(cells x n_grains) once.  Grains run in the colour-phase
 * kernels and the null-event form (the replica-resident kernel has no grain
 * tables), in both arithmetic forms and with site energies.
 * Errors: FKMC_EINVAL for bad parameters or a dimension shorter than
 * 2 width + 1; FKMC_ENOMEM (5 bytes per cell); FKMC_ECUDA. */
int kmc_set_grains(kmc_batch* b, const kmc_grains* g);

/* Grain of every cell (int32) and its boundary flag (uint8) for replica r,
 * cell index (z ny + y) nx + x; n must equal nx ny nz.  FKMC_ESTATE without
 * grains. */
int kmc_read_grains(kmc_batch* b, int32_t r, int32_t* grain, uint8_t* boundary, size_t n);

/* Run `windows` synchronisation windows on every replica.  Synchronous.
 * Errors: FKMC_ESTATE before kmc_set_barriers; FKMC_EOVERFLOW if a hand-off
 * found its target fragment full (the state is then invalid);
 * FKMC_ETIMEOUT if a device wait gave up; FKMC_ECUDA; FKMC_ESTATE if a site
 * energy difference fell outside the tables' bound (cannot happen for a
 * consistent field; the event was dropped). */
int kmc_run(kmc_batch* b, uint64_t windows, kmc_run_stats* stats);

/* The paper's own atom-based fragment kMC with null events (Sec. II.B,
 * Eqs. AtomP and TimeStepFrg), the atoms being the vacancies, for `steps`
 * steps on every replica.  One step:
 *   1. R_I = the sum of vacancy I's exchange rates, R_tot = sum_I R_I,
 *      R_max = max_I R_I, all exact u64 (rates in the fixed point of the mixed
 *      form with F_null = 63 - ceil(log2(8 N_V)), from the replica's fp32
 *      table);
 *   2. min(n_frg, N_V) distinct vacancies are picked: the images of
 *      0 .. N_frg-1 under a keyed bijection of the vacancy ids (an
 *      alternating Feistel network on ceil(log2 N_V) bits, four rounds
 *      x ^= fmix64(other half ^ k_r) with MurmurHash3's 64-bit finaliser, round
 *      keys the Philox block (step, 0, 0, 0) of (seed, replica), cycle
 *      walking back into [0, N_V));
 *   3. pick p draws x from Philox (step, p) and takes the first event whose
 *      running sum over the vacancy's 8 exchanges exceeds mulhi(x, R_max), or
 *      the null event when none does (probability 1 - R_I / R_max);
 *   4. a pick whose exchange shares a site with the exchange of a non-null
 *      pick of smaller index becomes null (the paper leaves the
 *      reconciliation of simultaneous picks open; this keeps the applied
 *      exchanges disjoint);
 *   5. the exchanges are applied, and the replica's clock advances by
 *      -ln(r') / R_tot * N_updated (r' from Philox (step, 2^64-1)).
 * With n_frg = 1 this is the conventional kMC of Sec. II.A in distribution.
 * The state is shared with kmc_run (records are regathered by id before and
 * returned to their fragments after); kmc_read_msd's t adds this clock.
 * Vacancy ids must be 0 .. N_V-1 (true after creation and kmc_write_state).
 * Needs 8 bytes per site (claims) and 24 bytes per vacancy of extra device
 * memory, allocated at the first call.
 * Errors: FKMC_ESTATE before kmc_set_barriers; FKMC_EINVAL for n_frg < 1,
 * more than 2^32 - 16 steps, or with site energies on; FKMC_ENOMEM;
 * FKMC_EOVERFLOW if a fragment cannot take its vacancies back (cap_v);
 * FKMC_ECUDA. */
int kmc_run_null(kmc_batch* b, uint64_t steps, int64_t n_frg, kmc_run_stats* stats);

/* Exact integer moments of the displacements of one species of replica r:
 * out = {count, sum dx, sum dy, sum dz, sum dx^2, sum dy^2, sum dz^2}, units
 * a/2 and (a/2)^2.  FKMC_V sums the vacancy records; FKMC_O / FKMC_H sum the
 * tracer field over the sites holding that species (FKMC_ESTATE without
 * tracer).  Computed by a reduction kernel into a small scratch buffer. */
int kmc_read_moments(kmc_batch* b, int32_t r, int32_t species, int64_t out[7]);

/* Vacancy moments of every replica in one reduction launch: out[7 r + k] as
 * in kmc_read_moments; n_out must be 7 x the number of replicas. */
int kmc_read_moments_all(kmc_batch* b, int64_t* out, size_t n_out);

/* Mean squared displacement per axis (m^2), mean displacement per axis (m)
 * and the simulated time t = windows * tau + the null-event clock (s) of one
 * species (Sec. III: D from tracked trajectories). */
int kmc_read_msd(kmc_batch* b, int32_t r, int32_t species, double msd_xyz[3],
                 double mean_xyz[3], double* t_s);

/* Diffusion coefficients of one species of replica r from the tracked
 * displacements after t = kmc_read_msd's time (Sec. III: D from the
 * trajectories of the particles; the bias run of the mu-scale model section):
 *   D_xyz[k]   = (<d_k^2> - <d_k>^2) / (2t)   per axis, the drift removed
 *                (D_z = D_xyz[2] along the field)                       m^2/s
 *   D          = (<dx^2> + <dy^2> + <dz^2>) / (6t)   MSD / (6t)           m^2/s
 *   D_xy       = (<dx^2> + <dy^2>) / (4t)    in the plane normal to the field
 *   v_drift[k] = <d_k> / t                   drift velocity               m/s
 * Means are over the replica's particles of that species, so the drift-removed
 * D_xyz needs many of them (with one particle it is 0).  Any output pointer
 * may be NULL.  Errors: as kmc_read_moments; FKMC_ESTATE before any simulated
 * time. */
int kmc_read_D(kmc_batch* b, int32_t r, int32_t species, double D_xyz[3], double* D, double* D_xy,
               double v_drift[3]);

/* Occupancy of replica r, one species code per site, site index
 * ((t nz + z) ny + y) nx + x with t the site type (0: a/2 x, 1: a/2 y,
 * 2: a/2 z from the cell corner).  n must equal 3 nx ny nz. */
int kmc_read_state(kmc_batch* b, int32_t r, uint8_t* host_occ, size_t n);

/* Replace the state of replica r: occupancy as given (codes 0..2), one record
 * per vacancy with zero displacement and id = rank in site order, tracer
 * field cleared, window counter kept.  Errors: FKMC_EINVAL for bad codes,
 * FKMC_EOVERFLOW if a fragment would exceed cap_v. */
int kmc_write_state(kmc_batch* b, int32_t r, const uint8_t* host_occ, size_t n);

/* Vacancy records of replica r as rows {fragment, site, dx, dy, dz, id},
 * fragments ascending and sites ascending inside a fragment.  *n_rows gets
 * the number of records; at most max_rows rows are written. */
int kmc_read_records(kmc_batch* b, int32_t r, int64_t* rows, int64_t max_rows, int64_t* n_rows);

/* Tracer displacements of replica r, 3 int32 per site (FKMC_ESTATE without tracer). */
int kmc_read_tracer(kmc_batch* b, int32_t r, int32_t* host_disp, size_t n_sites);

/* The whole mutable state of the batch as one opaque blob, for checkpoints
 * and end-to-end transfers: a header (magic, batch shape), per replica its
 * window and null-event step counters, hop and hand-off counters, null-event
 * clock and vacancy / H- counts, then the device arrays -- occupancy planes,
 * vacancy records and counts, and where present the tracer field, the dopants,
 * the electrostatic energies u and each replica's last potential (the warm
 * start of the next solve) with the windows since that solve.  A batch
 * created with the same cells, compositions, seed and options, given the same
 * kmc_set_barriers / kmc_set_site_energy / kmc_set_grains /
 * kmc_set_electrostatics calls, continues from an uploaded blob exactly as
 * the batch it was downloaded from (the random streams are keyed by the
 * restored counters).  kmc_state_bytes gives the size; kmc_download_state /
 * kmc_upload_state copy it to / from host memory (pinned memory gives full
 * copy bandwidth).  Errors: FKMC_EINVAL for a wrong size or a blob of another
 * batch shape (replica count, sizes, cap_v, tracer, dopants, electrostatics
 * on/off); FKMC_ECUDA. */
int kmc_state_bytes(kmc_batch* b, size_t* bytes);
int kmc_download_state(kmc_batch* b, void* host, size_t bytes);
int kmc_upload_state(kmc_batch* b, const void* host, size_t bytes);

int kmc_get_replica_info(kmc_batch* b, int32_t r, kmc_replica_info* out);

/* Invariant check of replica r's device state, for debugging and tests.  Every
 * event of the fragment BKL exchanges a vacancy with a neighbouring ion
 * (Sec. II.A, Eqs. eventSelection and TimeStep), so the counts of vacancies
 * and of H- ions never change, and the vacancy records must describe the
 * occupancy exactly.  Two kernels on the batch's stream measure, without
 * copying the lattice to the host:
 *   sites[code]        occupancy census by code (FKMC_O, FKMC_H, FKMC_V; 3 is
 *                      unused and must be 0);
 *   records            records over all fragment lists;
 *   rec_not_vacancy    records whose site does not hold a vacancy;
 *   rec_wrong_fragment records listed by a fragment that does not own the site;
 *   rec_outside        records whose site lies outside the lattice;
 *   frag_bad_count     fragments whose count is below 0 or above cap_v;
 *   hash_vac_sites, hash_rec_sites  sums (mod 2^64) of a 64-bit mixing
 *                      function of the linear site index over the vacancy
 *                      sites and over the record sites: equal sums with equal
 *                      counts mean one record per vacancy site (up to a 2^-64
 *                      chance of a collision);
 *   hash_rec_ids, hash_ids_expected the same sum over the record ids and over
 *                      0 .. n_vac-1 (each vacancy keeps its id).
 * ok = 1 when the counts equal the replica's vacancies and H- ions and every
 * check holds.  Synchronous (waits for the batch's stream); the first call
 * allocates 96 bytes through the batch's allocator.  Check after every window
 * by running one window per kmc_run call.  Errors: FKMC_EINVAL for a bad
 * replica or a NULL output, FKMC_ENOMEM, FKMC_ECUDA. */
typedef struct {
    int64_t sites[4];
    int64_t records, rec_not_vacancy, rec_wrong_fragment, rec_outside, frag_bad_count;
    uint64_t hash_vac_sites, hash_rec_sites, hash_rec_ids, hash_ids_expected;
    int32_t ok;
    int32_t pad;
} kmc_invariants;
int kmc_check_invariants(kmc_batch* b, int32_t r, kmc_invariants* out);
int32_t kmc_num_replicas(const kmc_batch* b);

/* Host-only: the rate table of kmc_set_barriers for one parameter set. */
int kmc_rate_table(const kmc_barrier_table* t, double T_K, double field_z_Vpm, double a_angstrom,
                   int32_t cap_v, double k64[6], float k32[6], uint64_t q[6], int32_t* F);

/* Host-only: fragments along one dimension of L cells for a target fragment
 * edge (what kmc_create_batch uses where kmc_opts.nfrag[d] == 0).  The paper
 * cuts a lattice into fragments without fixing their number; the reading: the
 * even count nearest L / edge (half-way cases up), but at least 2, reduced
 * while a fragment would be shorter than 2 cells; 1 for L < 4.  Edges are then
 * floor(L / n) or floor(L / n) + 1.  Returns 0 for L < 1 or edge < 1. */
int32_t kmc_partition_count(int32_t L, int32_t edge);

/* Host-only: the 8 neighbours of each site type as rows {t2, dcx, dcy, dcz,
 * dx, dy, dz} (24 rows of int32): neighbour cell offset and displacement in
 * units of a/2, ascending in (dx, dy, dz). */
void kmc_neighbour_table(int32_t out[168]);

/* Allocation-free variant of kmc_read_moments_all.  The paper has no
 * counterpart: this is a service for callers that cannot allocate device
 * memory -- a host framework that owns every device allocation through its
 * own pool, a plugin that is handed fixed buffers, a serving loop whose memory
 * is planned ahead.  The caller passes its own device buffers and gets the
 * moments back; the library calls no cudaMalloc, cudaFree or allocating
 * routine here.
 *   d_records        device array of offsets[n_groups] x cap_v 24-byte records
 *                    {u64 site key, int32 d[3], uint32 id} (the batch's layout),
 *                    fragment-major; only the displacements d are read; it must
 *                    hold offsets[n_groups] x cap_v records on the current device
 *   d_counts         device int32[offsets[n_groups]]: slots in use per fragment
 *                    (each <= cap_v), on the current device
 *   fragment_offsets host int64[n_groups + 1]: group g owns fragments
 *                    [offsets[g], offsets[g+1]); offsets[0] = 0, non-decreasing
 *                    (a group may be empty); offsets[n_groups] x cap_v must fit
 *                    in int64
 *   n_groups         1 .. FKMC_NOALLOC_MAX_GROUPS
 *   out              host int64[7 n_groups], as in kmc_read_moments
 *   stream           cudaStream_t (NULL = legacy default stream)
 * The call is synchronous (it waits for the stream and copies into `out`), so
 * it must not be made while its stream is being captured: it then returns
 * FKMC_EINVAL.  Its only scratch (the offsets and the accumulators, about
 * 256 KiB) is a static device array that every GPU loading the library holds
 * until the process exits.  The first call on a device looks up that array's
 * address (cudaGetSymbolAddress) and the SM count with the device current.
 * All calls share the array and it keeps the last call's contents (the
 * accumulators are cleared at the start of each call), so calls that overlap
 * on the GPU -- on two streams, or from two threads -- race.
 * Errors: FKMC_EINVAL for null pointers, n_groups outside [1, 4096], cap_v
 * outside [1, 256], bad offsets or a capturing stream; FKMC_ECUDA. */
#define FKMC_NOALLOC_MAX_GROUPS 4096
int kmc_vacancy_moments_noalloc(const void* d_records, const int32_t* d_counts,
                                const int64_t* fragment_offsets, int32_t n_groups, int32_t cap_v,
                                int64_t* out, void* stream);

int kmc_destroy(kmc_batch* b);

const char* kmc_last_error(void);

#ifdef __cplusplus
}
#endif

#endif
