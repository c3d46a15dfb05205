// fkmc_api.cu -- host side of the C ABI declared in include/fkmc.h:
// validation, partition of the lattice into fragments, device buffers,
// rate tables (Eq. RateCnst1 of arXiv:2004.09081 with the ESP shift of
// Sec. III), the window loop and the read-outs.
#include <cuda_runtime.h>
#include <nvtx3/nvToolsExt.h>

#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <string>
#include <vector>

#include "fkmc.h"
#include "fkmc_check.h"
#include "fkmc_kernels.h"

namespace {
// NVTX range over one ABI call, named after it (shown by Nsight tools; without
// a tool attached the header-only NVTX calls do nothing)
struct NvtxRange {
    explicit NvtxRange(const char* name) { nvtxRangePushA(name); }
    ~NvtxRange() { nvtxRangePop(); }
    NvtxRange(const NvtxRange&) = delete;
    NvtxRange& operator=(const NvtxRange&) = delete;
};
}  // namespace

using namespace fkmc;

namespace {

thread_local std::string g_err;

int fail(int code, const std::string& msg)
{
    g_err = msg;
    return code;
}

int cuda_fail(cudaError_t e, const char* what)
{
    return fail(FKMC_ECUDA, std::string(what) + ": " + cudaGetErrorString(e));
}

#define CK(call, what)                                  \
    do {                                                \
        cudaError_t e_ = (call);                        \
        if (e_ != cudaSuccess) return cuda_fail(e_, what); \
    } while (0)

const double KB_EV = 8.617333262e-5;  // Boltzmann constant, eV/K (R of Eq. RateCnst1)

// Neighbour table built from the geometry: a site of type t sits at a/2 e_t
// from its cell corner; its 8 nearest O neighbours are at a/2 (s_t e_t + s_u e_u)
// for the two other axes u and signs s_t, s_u = +-1.  The neighbour has type u
// and lies in the cell offset (d + e_t - e_u)/2.  Listed in ascending (dx,dy,dz).
void build_nb_table(NbEntry tab[3][8])
{
    for (int t = 0; t < 3; ++t) {
        struct Row { int d[3]; int u; };
        std::vector<Row> rows;
        for (int u = 0; u < 3; ++u) {
            if (u == t) continue;
            for (int st = -1; st <= 1; st += 2)
                for (int su = -1; su <= 1; su += 2) {
                    Row r{};
                    r.d[t] = st;
                    r.d[u] = su;
                    r.u = u;
                    rows.push_back(r);
                }
        }
        std::sort(rows.begin(), rows.end(), [](const Row& a, const Row& b) {
            return std::lexicographical_compare(a.d, a.d + 3, b.d, b.d + 3);
        });
        for (int n = 0; n < 8; ++n) {
            NbEntry& e = tab[t][n];
            e.t2 = (int8_t)rows[n].u;
            for (int k = 0; k < 3; ++k) {
                e.d[k] = (int8_t)rows[n].d[k];
                e.dc[k] = (int8_t)((rows[n].d[k] + (k == t) - (k == rows[n].u)) / 2);
            }
            e.pad = 0;
        }
    }
}

int partition_count(int L, int edge)
{
    int nf = 2 * (int)std::floor((double)L / (2.0 * edge) + 0.5);
    if (nf < 2) nf = L >= 4 ? 2 : 1;
    while (nf > 1 && L / nf < 2) nf -= 2;
    if (nf < 1) nf = 1;
    return nf;
}

bool partition_ok(int L, int nf)
{
    if (nf < 1 || nf > L) return false;
    if (nf == 1) return true;
    return (nf % 2 == 0) && (L / nf >= 2);
}

int ceil_log2(int64_t v)
{
    int lg = 0;
    while (((int64_t)1 << lg) < v) ++lg;
    return lg;
}

}  // namespace

namespace fkmc {
// error reporting shared with the other translation units of the library
int set_error(int code, const char* msg)
{
    return fail(code, msg);
}
}  // namespace fkmc

struct kmc_batch {
    int n = 0;
    kmc_opts opts{};
    cudaStream_t st = nullptr;
    int cap = 0;
    std::vector<RepDesc> desc;
    std::vector<int64_t> n_vac, n_H;
    std::vector<int> b_bits;
    std::vector<double> a_ang;
    std::vector<unsigned long long> stats_host;  // hops, handoffs per replica
    int64_t nfrag_total = 0, occ_words = 0, nsite_total = 0, total_items = 0;
    bool rates_set = false;
    // device buffers
    uint32_t* occ = nullptr;
    VacRec* recs = nullptr;
    int32_t* counts = nullptr;
    int32_t* tracer = nullptr;
    RepDesc* d_desc = nullptr;
    unsigned long long* stats = nullptr;
    uint32_t* status = nullptr;
    unsigned long long* scratch = nullptr;  // 7 moments
    unsigned long long* scratch_all = nullptr;  // 7 moments per replica
    unsigned long long* check_buf = nullptr;    // CHECK_WORDS sums of kmc_check_invariants
    cudaEvent_t ev0 = nullptr, ev1 = nullptr;
    std::vector<void*> owned;
    // replica-resident kernel: replicas grouped by shared-memory size class
    NbTable nbt{};
    int32_t* d_reps = nullptr;   // resident replica ids, class by class
    ClusterPlan* d_plans = nullptr;  // cluster-resident replicas' slab plans, grouped by CTA count
    ResCache rcache{};               // fragment totals the resident kernels carry from call to call
    int64_t* d_nvac = nullptr;   // vacancies per replica
    // a launch of the replica-resident kernel (one CTA, or a 2-CTA mirrored pair, per
    // replica; start/count index d_reps) or of the cluster-resident kernel (slabs
    // == true: one cluster of `cluster` CTAs per replica; start/count index d_plans)
    struct RClass {
        int start, count;
        size_t smem;
        int threads;
        int cluster;
        cudaStream_t st;
        cudaEvent_t done;
        bool slabs;
    };
    std::vector<RClass> rclass;
    cudaEvent_t fork = nullptr;
    cudaGraphExec_t res_exec = nullptr;  // one call's class launches (fork, launches, join), captured
    uint64_t res_exec_windows = 0;
    cudaStream_t res_st = nullptr;       // the graph's stream, beside the colour-phase launches
    cudaEvent_t res_fork = nullptr, res_join = nullptr;
    cudaStream_t side_st = nullptr;       // the small-fragment run pass, beside the general one
    cudaEvent_t side_fork = nullptr, side_join = nullptr;
    bool any_global = true;
    int cluster_top = 0;  // how many of the largest replicas run as 2-CTA clusters (kmc_opts)
    std::vector<int32_t> run_kernel, run_ctas;  // per replica: kmc_replica_info.kernel and .ctas
    // colour-phase path: per-window set-up, screen and run, captured once in a graph
    unsigned long long* wctl = nullptr;  // [0] windows of this call so far, [1] current offset
    uint32_t* perms = nullptr;           // colour order of every replica, this window
    ActEntry* act = nullptr;             // screened fragments of a phase
    int32_t* act_count = nullptr;        // per list and phase
    uint8_t* cls = nullptr;              // per work item: the screen's class for the register lane pass
    int run_blocks = 0;
    cudaStream_t cap_st = nullptr;
    cudaGraphExec_t window_exec = nullptr;
    // site-energy interactions (plain form, colour-phase kernels)
    bool site_on = false;
    bool field_valid = false;
    std::vector<int64_t> n_fe;
    std::vector<double> T;           // temperature of every replica (kmc_set_barriers)
    int n_vv = 0, n_bo = 0, e_self = 0;
    int64_t e_bound = 0;             // bound on |E_site|, 1e-4 eV units
    int64_t ncell_total = 0;
    uint8_t* fe = nullptr;           // one byte per cell, batch-wide cell index
    int32_t* field = nullptr;        // E_site per O site
    SiteOff* d_vv = nullptr;
    SiteOff* d_bo = nullptr;
    double* btab = nullptr;          // Boltzmann tables of every replica
    size_t btab_bytes = 0;
    // electrostatics (mu-scale model): potential of the vacancy charges, frozen between refreshes
    bool elec_on = false;
    kmc_electrostatics elec{};
    int32_t* elec_u = nullptr;          // q phi per O site, 1e-4 eV units (batch-wide site index)
    int32_t* d_elec_g = nullptr;        // [replica][3][8] own-potential share of a hop
    std::vector<int32_t> elec_g;        // host copy
    unsigned* d_umax = nullptr;         // max |u| of the last refresh
    int64_t elec_umax = 0;
    uint64_t elec_age = 0;              // windows since the last refresh
    MgPlan mg{};
    MgBuffers mgb{};
    int64_t mg_total = -1, mg_nodes = -1;
    double* phi_prev = nullptr;         // each replica's last potential (warm start of the next solve)
    struct ElecGraph {                  // one refresh solve + update of replica r, captured
        int r, cycles;
        bool warm, field;
        cudaGraphExec_t exec;
    };
    std::vector<ElecGraph> elec_graphs;
    bool phi_prev_valid = false;
    // grains (mu-scale model): boundary cells raise the barrier of hops touching them
    bool grains_on = false;
    kmc_grains grains{};
    int32_t* grain = nullptr;              // grain of every cell
    uint8_t* gbound = nullptr;             // boundary flag of every cell
    int64_t* gX = nullptr;                 // seed positions
    int64_t gX_len = 0;
    std::vector<kmc_barrier_table> tables; // of the last kmc_set_barriers
    std::vector<double> Ez;
    // atom-based fragment kMC with null events (Sec. II.B)
    VacRec* vac = nullptr;                 // vacancies by id, replica after replica
    int64_t vac_cap = 0;
    unsigned long long* claims = nullptr;  // per site: (step tag, pick) of the earliest claim
    NullProp* props = nullptr;
    int64_t props_cap = 0;
    unsigned long long* nacc = nullptr;    // R_tot, R_max, N_updated per replica
    double* theta = nullptr;               // null-event clock per replica (1/k32max units)
    double* nE = nullptr;                  // the current step's clock variate per replica
    unsigned long long* nctl = nullptr;    // [0] steps of this call so far, [1] current step, [2] blocks done
    std::vector<double> theta_host;
    cudaGraphExec_t null_exec = nullptr;
    int64_t null_exec_picks = -1, null_exec_vac = -1;
    bool null_exec_grains = false;

    void* dalloc(size_t bytes)
    {
        bytes = (bytes + 255) & ~(size_t)255;
        if (bytes == 0) bytes = 256;
        void* p = nullptr;
        if (opts.alloc) {
            p = opts.alloc(opts.alloc_ctx, bytes);
        } else if (cudaMalloc(&p, bytes) != cudaSuccess) {
            cudaGetLastError();
            p = nullptr;
        }
        if (p) owned.push_back(p);
        return p;
    }

    void dfree(void* p)
    {
        if (!p) return;
        auto it = std::find(owned.begin(), owned.end(), p);
        if (it == owned.end()) return;
        owned.erase(it);
        if (opts.alloc) {
            if (opts.free) opts.free(opts.alloc_ctx, p);
        } else {
            cudaFree(p);
        }
    }

    void release()
    {
        for (void* p : owned) {
            if (opts.alloc) {
                if (opts.free) opts.free(opts.alloc_ctx, p);
            } else {
                cudaFree(p);
            }
        }
        owned.clear();
        if (ev0) cudaEventDestroy(ev0);
        if (ev1) cudaEventDestroy(ev1);
        if (fork) cudaEventDestroy(fork);
        ev0 = ev1 = fork = nullptr;
        if (side_fork) cudaEventDestroy(side_fork);
        if (side_join) cudaEventDestroy(side_join);
        if (side_st) cudaStreamDestroy(side_st);
        side_fork = side_join = nullptr;
        side_st = nullptr;
        for (auto& c : rclass) {
            if (c.st) cudaStreamDestroy(c.st);
            if (c.done) cudaEventDestroy(c.done);
        }
        rclass.clear();
        if (window_exec) cudaGraphExecDestroy(window_exec);
        if (res_exec) cudaGraphExecDestroy(res_exec);
        res_exec = nullptr;
        if (res_st) cudaStreamDestroy(res_st);
        if (res_fork) cudaEventDestroy(res_fork);
        if (res_join) cudaEventDestroy(res_join);
        res_st = nullptr;
        res_fork = res_join = nullptr;
        if (null_exec) cudaGraphExecDestroy(null_exec);
        null_exec = nullptr;
        for (auto& g : elec_graphs) cudaGraphExecDestroy(g.exec);
        elec_graphs.clear();
        if (cap_st) cudaStreamDestroy(cap_st);
        window_exec = nullptr;
        cap_st = nullptr;
    }
};

namespace {

// the site-energy run pass is on: shells, dopant energies or electrostatics
bool site_path(const kmc_batch* b) { return b->site_on || b->elec_on; }

// anything but a resident run changed a replica's state or rates: the resident
// kernels' fragment totals from the last call no longer hold
int drop_resident_cache(kmc_batch* b)
{
    if (b->rcache.valid) CK(cudaMemsetAsync(b->rcache.valid, 0, (size_t)b->n, b->st), "memset");
    return FKMC_OK;
}

// kernel launches of one window of the colour-phase path: set-up, then per phase
// screen + run, + the grouped small pass where it runs, or the one-thread-per-
// fragment pass + run
uint64_t window_launches(const kmc_batch* b)
{
    const bool split = window_split(site_path(b), b->total_items, b->opts.small_pass);
    return split && window_lane(b->opts.precision, b->opts.small_pass, b->opts.lane_form, b->total_items) !=
                        LANE_PERSISTENT
               ? 25
               : 17;
}

int check_status(kmc_batch* b)
{
    uint32_t s = 0;
    CK(cudaMemcpyAsync(&s, b->status, sizeof s, cudaMemcpyDeviceToHost, b->st), "status copy");
    CK(cudaStreamSynchronize(b->st), "synchronize");
    if (s & STATUS_OVERFLOW)
        return fail(FKMC_EOVERFLOW, "a fragment received more vacancies than cap_v slots");
    if (s & STATUS_TIMEOUT) return fail(FKMC_ETIMEOUT, "a device-side wait ran out of time");
    if (s & STATUS_EVENT_LIMIT)
        return fail(FKMC_ETIMEOUT, "a fragment reached the per-phase event limit (window too long)");
    if (s & STATUS_ENERGY_RANGE)
        return fail(FKMC_ESTATE, "a site-energy difference fell outside the Boltzmann tables' bound");
    return FKMC_OK;
}

int upload_desc(kmc_batch* b)
{
    CK(cudaMemcpyAsync(b->d_desc, b->desc.data(), sizeof(RepDesc) * b->n, cudaMemcpyHostToDevice, b->st),
       "descriptor upload");
    CK(cudaStreamSynchronize(b->st), "synchronize");
    return FKMC_OK;
}

int rate_table_impl(const kmc_barrier_table* t, double T_K, double Ez, double a_ang, int cap_v,
                    double k64[6], float k32[6], uint64_t q[6], int32_t* F_out)
{
    if (!t || !(T_K > 0.0) || !std::isfinite(T_K) || !std::isfinite(Ez) || !(a_ang > 0.0) ||
        !std::isfinite(t->Ea_O_eV) || !std::isfinite(t->Ea_H_eV) || !(t->prefactor > 0.0) ||
        !std::isfinite(t->q_O) || !std::isfinite(t->q_H) || cap_v < 1)
        return fail(FKMC_EINVAL, "rate table: T must be > 0, inputs finite, prefactor > 0");
    const double Ea[2] = {t->Ea_O_eV, t->Ea_H_eV};
    const double qc[2] = {t->q_O, t->q_H};
    const double half_a_m = 0.5 * a_ang * 1e-10;
    for (int h = 0; h < 2; ++h)
        for (int dz = -1; dz <= 1; ++dz) {
            // Eq. (RateCnst1) with the vacancy's z step dz a/2 shifting the barrier by dU/2
            const double dz_m = (double)dz * half_a_m;
            const double dU = -(qc[h] * Ez) * dz_m;
            const double barrier = Ea[h] + 0.5 * dU;
            k64[3 * h + dz + 1] = t->prefactor * std::exp(-(barrier / (KB_EV * T_K)));
        }
    float kmax = 0.0f;
    for (int i = 0; i < 6; ++i) {
        k32[i] = (float)k64[i];
        kmax = std::max(kmax, k32[i]);
    }
    if (!(kmax > 0.0f) || !std::isfinite(kmax))
        return fail(FKMC_EINVAL, "rate table: rates underflow or overflow in fp32");
    const int F = 63 - ceil_log2(8 * (int64_t)cap_v);
    for (int i = 0; i < 6; ++i) q[i] = (uint64_t)std::llrint(std::ldexp((double)k32[i] / (double)kmax, F));
    *F_out = F;
    return FKMC_OK;
}

bool valid_replica(const kmc_batch* b, int32_t r) { return b && r >= 0 && r < b->n; }

// Decide which replicas run in the replica-resident kernel and group them
// into shared-memory size classes (one launch per class, on forked streams).
int plan_residency(kmc_batch* b)
{
    if (int rc0 = drop_resident_cache(b)) return rc0;
    if (b->res_exec) cudaGraphExecDestroy(b->res_exec);  // it holds the old classes' launches
    b->res_exec = nullptr;
    for (auto& c : b->rclass) {
        if (c.st) cudaStreamDestroy(c.st);
        if (c.done) cudaEventDestroy(c.done);
    }
    b->rclass.clear();
    const bool allowed = b->opts.precision == FKMC_MIXED && b->opts.schedule != 1 &&
                         b->cap <= RESIDENT_MAX_SLOTS && !site_path(b) && !b->grains_on;
    // launch classes: (shared-memory bound, threads); a replica takes the first
    // class its state fits, so small replicas pack several CTAs per SM and the
    // largest get the most warps that still fit beside their state.  The
    // `cluster_top` largest replicas of the 1024-thread class run as 2-CTA
    // clusters (two SMs each), as long as the GPU has the SMs to spare.
    const size_t bounds[5] = {24 * 1024, 48 * 1024, 96 * 1024, RESIDENT_MAX_SMEM, RESIDENT_MAX_SMEM};
    const int threads[5] = {128, 128, 256, 1024, 512};
    std::vector<std::vector<int>> cls(6);
    std::vector<size_t> cmax(6, 0), need_of(b->n, 0);
    std::vector<ClusterPlan> plans;
    b->any_global = false;
    b->run_kernel.assign(b->n, 0);
    b->run_ctas.assign(b->n, 0);
    for (int r = 0; r < b->n; ++r) {
        int c = -1;
        size_t need = 0;
        for (int k = 0; k < 5 && allowed && c < 0; ++k) {
            need = resident_smem_bytes(b->desc[r], b->n_vac[r], b->cap, threads[k], 1, 2);
            if (need <= bounds[k]) c = k;
        }
        // the first draws of as many colour phases per batch as the class's shared
        // memory allows beside the state (8: one batch per window): four events per
        // fragment where 2 or more phases of them fit, else two
        b->desc[r].pre_g = 1;
        b->desc[r].pre_ev = 2;
        static const int pick[6][2] = {{8, 4}, {4, 4}, {2, 4}, {8, 2}, {4, 2}, {2, 2}};  // (phases, events)
        for (int k = 0; c >= 0 && k < 6; ++k) {
            const size_t ng = resident_smem_bytes(b->desc[r], b->n_vac[r], b->cap, threads[c], pick[k][0], pick[k][1]);
            if (ng <= bounds[c]) {
                b->desc[r].pre_g = pick[k][0];
                b->desc[r].pre_ev = pick[k][1];
                need = ng;
                break;
            }
        }
        // the cluster-resident kernel: a replica too large for one SM (or every
        // replica, with cluster_ctas forced) held by a cluster of CTAs, one z-slab each
        const int force = b->opts.cluster_ctas;
        if (allowed && force >= 0 && (c < 0 || force >= 2)) {
            ClusterPlan pl{};
            const int lo = force >= 2 ? force : 2, hi = force >= 2 ? force : CLUSTER_MAX_CTAS;
            if (make_cluster_plan(b->desc[r], b->n_vac[r], b->cap, lo, hi, &pl) &&
                cluster_fits(pl.ncta, cluster_smem_bytes(b->desc[r], pl, b->cap)) > 0) {
                pl.rep = r;
                plans.push_back(pl);
                b->desc[r].resident = 1;
                b->run_kernel[r] = 2;
                b->run_ctas[r] = pl.ncta;
                continue;
            }
        }
        b->desc[r].resident = c >= 0 ? 1 : 0;
        if (c < 0) {
            b->any_global = true;
            continue;
        }
        cls[c].push_back(r);
        need_of[r] = need;
        b->run_kernel[r] = 1;
        b->run_ctas[r] = 1;
    }
    // largest replicas (by vacancies, the work per phase) first in every class: the
    // longest-running CTAs start earliest, which shortens the tail of the launch
    for (int c = 0; c < 5; ++c)
        std::sort(cls[c].begin(), cls[c].end(), [&](int a, int q) {
            return b->n_vac[a] != b->n_vac[q] ? b->n_vac[a] > b->n_vac[q] : a < q;
        });
    // optionally the largest of the 1024-thread class run as 2-CTA clusters (class 5)
    const int ntop = std::min<int>((int)cls[3].size(), b->cluster_top);
    cls[5].assign(cls[3].begin(), cls[3].begin() + ntop);
    cls[3].erase(cls[3].begin(), cls[3].begin() + ntop);
    for (int r : cls[5]) b->run_ctas[r] = 2;
    for (int c = 0; c < 6; ++c)
        for (int r : cls[c]) cmax[c] = std::max(cmax[c], need_of[r]);
    if (b->opts.schedule == 2 && b->any_global)
        return fail(FKMC_EINVAL, "schedule 2 needs every replica to fit the resident kernel (mixed form)");
    std::vector<int32_t> order;
    for (int c = 0; c < 6; ++c) {
        if (cls[c].empty()) continue;
        kmc_batch::RClass rc{(int)order.size(), (int)cls[c].size(), cmax[c], c == 5 ? 1024 : threads[c],
                             c == 5 ? 2 : 1, nullptr, nullptr, false};
        for (int r : cls[c]) order.push_back(r);
        CK(cudaStreamCreateWithFlags(&rc.st, cudaStreamNonBlocking), "stream");
        CK(cudaEventCreateWithFlags(&rc.done, cudaEventDisableTiming), "event");
        b->rclass.push_back(rc);
    }
    if (!order.empty())
        CK(cudaMemcpyAsync(b->d_reps, order.data(), sizeof(int32_t) * order.size(), cudaMemcpyHostToDevice,
                           b->st),
           "replica list upload");
    // cluster-resident replicas: one launch per CTA count (a launch has one cluster shape)
    std::stable_sort(plans.begin(), plans.end(),
                     [](const ClusterPlan& x, const ClusterPlan& y) { return x.ncta < y.ncta; });
    for (size_t k = 0; k < plans.size();) {
        size_t e = k, smem = 0;
        while (e < plans.size() && plans[e].ncta == plans[k].ncta) {
            smem = std::max(smem, cluster_smem_bytes(b->desc[plans[e].rep], plans[e], b->cap));
            ++e;
        }
        kmc_batch::RClass rc{(int)k, (int)(e - k), smem, CLUSTER_THREADS, plans[k].ncta, nullptr, nullptr, true};
        CK(cudaStreamCreateWithFlags(&rc.st, cudaStreamNonBlocking), "stream");
        CK(cudaEventCreateWithFlags(&rc.done, cudaEventDisableTiming), "event");
        b->rclass.push_back(rc);  // launched last-first: a cluster takes its SMs before single CTAs spread out
        k = e;
    }
    if (!plans.empty())
        CK(cudaMemcpyAsync(b->d_plans, plans.data(), sizeof(ClusterPlan) * plans.size(), cudaMemcpyHostToDevice,
                           b->st),
           "cluster plan upload");
    return FKMC_OK;
}

// ---------------------------------------------------------------- site energies
// Partners of a site by displacement: a vector d (units a/2) from a site at p0
// lands on an O site when exactly one coordinate of p0 + d is odd (that axis is
// the O site's type), on a B site (cell corner) when all are even.
struct Landing { int kind; int t2; int dc[3]; };  // kind 0: O site, 1: B site, -1: neither

Landing land(const int p0[3], const int d[3])
{
    Landing L{-1, -1, {0, 0, 0}};
    int p[3], odd = 0, axis = -1;
    for (int k = 0; k < 3; ++k) {
        p[k] = p0[k] + d[k];
        if (p[k] & 1) { ++odd; axis = k; }
    }
    if (odd == 1) {
        L.kind = 0;
        L.t2 = axis;
        for (int k = 0; k < 3; ++k) L.dc[k] = (p[k] - (k == axis)) / 2;
    } else if (odd == 0) {
        L.kind = 1;
        for (int k = 0; k < 3; ++k) L.dc[k] = p[k] / 2;
    }
    return L;
}

int32_t energy_units(double eV) { return (int32_t)std::llrint(eV * 1e4); }

// Partner tables of a shell set: V-V partners of each O site type, the O
// sites around a B site (dopant scatter), the B sites around each O site type,
// the reaches in cells, the bound on |E_site| and the a/sqrt2 shell energy.
struct ShellTables {
    std::vector<SiteOff> vv = std::vector<SiteOff>((size_t)3 * SITE_MAX_VV);
    int nvv = 0;
    std::vector<SiteOff> bo;
    std::vector<SiteOff> ob[3];
    int reach_vv = 0, reach_all = 0;
    int64_t bound = 0;
    int32_t e_self = 0;
};

int make_shells(const kmc_site_energy* e, ShellTables* out)
{
    if (e->n_vv < 0 || e->n_vv > FKMC_MAX_SHELLS || e->n_fe < 0 || e->n_fe > FKMC_MAX_SHELLS)
        return fail(FKMC_EINVAL, "0 to 8 shells of each kind");
    const int ns = e->n_vv + e->n_fe;
    auto d2_of = [&](int k) { return k < e->n_vv ? e->vv_d2[k] : e->fe_d2[k - e->n_vv]; };
    auto en_of = [&](int k) { return k < e->n_vv ? e->vv_eV[k] : e->fe_eV[k - e->n_vv]; };
    for (int k = 0; k < ns; ++k) {
        if (d2_of(k) < 1 || d2_of(k) > 36 || !std::isfinite(en_of(k)) || std::fabs(en_of(k)) > 10.0)
            return fail(FKMC_EINVAL, "shell squared distances must be in [1, 36], energies finite within 10 eV");
        for (int q = 0; q < k; ++q)
            if ((q < e->n_vv) == (k < e->n_vv) && d2_of(q) == d2_of(k))
                return fail(FKMC_EINVAL, "a shell is listed twice");
    }
    ShellTables& sh = *out;
    int nvv[3] = {0, 0, 0};
    std::vector<int> hit(ns, 0);
    // centre = an O site of type t (t = 0..2) or a B site (t = 3); |d| <= 6
    // half-units per axis covers every squared distance up to 36
    for (int t = 0; t < 4; ++t) {
        const int p0[3] = {t == 0, t == 1, t == 2};
        int64_t sum = 0;
        for (int dz = -6; dz <= 6; ++dz)
            for (int dy = -6; dy <= 6; ++dy)
                for (int dx = -6; dx <= 6; ++dx) {
                    const int d[3] = {dx, dy, dz};
                    const int d2 = dx * dx + dy * dy + dz * dz;
                    const Landing L = land(p0, d);
                    if (L.kind < 0) continue;
                    // O centre: O partners in V-V shells, B partners in dopant shells;
                    // B centre: O partners in dopant shells
                    const bool want_vv = t < 3 && L.kind == 0;
                    if (!want_vv && (L.kind == 0) == (t < 3)) continue;
                    for (int k = want_vv ? 0 : e->n_vv; k < (want_vv ? e->n_vv : ns); ++k) {
                        if (d2_of(k) != d2) continue;
                        hit[k] = 1;
                        SiteOff o;
                        o.t2 = (int8_t)(L.kind == 0 ? L.t2 : -1);
                        for (int a = 0; a < 3; ++a) o.dc[a] = (int8_t)L.dc[a];
                        o.e = energy_units(en_of(k));
                        int reach = 0;
                        for (int a = 0; a < 3; ++a) reach = std::max(reach, std::abs(L.dc[a]));
                        sh.reach_all = std::max(sh.reach_all, reach);
                        if (t == 3) {
                            if ((int)sh.bo.size() == SITE_MAX_BO) return fail(FKMC_EINVAL, "too many dopant partners");
                            sh.bo.push_back(o);
                            continue;
                        }
                        sum += o.e < 0 ? -(int64_t)o.e : o.e;
                        if (want_vv) {
                            sh.reach_vv = std::max(sh.reach_vv, reach);
                            if (nvv[t] == SITE_MAX_VV) return fail(FKMC_EINVAL, "too many V-V partners per site");
                            sh.vv[(size_t)t * SITE_MAX_VV + nvv[t]++] = o;
                        } else {
                            sh.ob[t].push_back(o);
                        }
                    }
                }
        if (t < 3) sh.bound = std::max(sh.bound, sum);
    }
    for (int k = 0; k < ns; ++k)
        if (!hit[k]) return fail(FKMC_EINVAL, "a squared distance is not a shell of this lattice");
    sh.nvv = nvv[0];
    for (int k = 0; k < e->n_vv; ++k)
        if (e->vv_d2[k] == 2) sh.e_self = energy_units(e->vv_eV[k]);
    return FKMC_OK;
}

// bound on |E_site| over every site: shells plus the electrostatic term
int64_t energy_bound(const kmc_batch* b)
{
    int64_t g = 0;
    for (int32_t v : b->elec_g) g = std::max<int64_t>(g, v < 0 ? -(int64_t)v : v);
    return b->e_bound + (b->elec_on ? b->elec_umax + g : 0);
}

// Boltzmann tables of every replica: lo[m0] = exp(-m0 c), hi[i] = exp(-512 (i - mid) c),
// c = 1e-4 / (2 kB T); |m| <= 2 e_bound, so m >> 9 stays within [-mid, mid].
int build_btab(kmc_batch* b)
{
    const int mid = (int)((2 * energy_bound(b) + 511) / 512) + 1;
    const int len = 2 * mid + 1;
    const size_t per = (size_t)BOLTZ_LO + len;
    std::vector<double> h(per * b->n);
    for (int r = 0; r < b->n; ++r) {
        const double c = 1e-4 / (2.0 * (KB_EV * b->T[r]));
        double* lo = h.data() + per * r;
        for (int m0 = 0; m0 < BOLTZ_LO; ++m0) lo[m0] = std::exp(-((double)m0 * c));
        for (int i = 0; i < len; ++i) lo[BOLTZ_LO + i] = std::exp(-((double)(512 * (int64_t)(i - mid)) * c));
        b->desc[r].btab_off = (int64_t)(per * r);
        b->desc[r].bhi_mid = mid;
        b->desc[r].bhi_len = len;
    }
    const size_t bytes = sizeof(double) * h.size();
    if (bytes > b->btab_bytes) {
        b->dfree(b->btab);
        b->btab = (double*)b->dalloc(bytes);
        b->btab_bytes = b->btab ? bytes : 0;
        if (!b->btab) return fail(FKMC_ENOMEM, "device allocation failed (Boltzmann tables)");
    }
    CK(cudaMemcpyAsync(b->btab, h.data(), bytes, cudaMemcpyHostToDevice, b->st), "table upload");
    CK(cudaStreamSynchronize(b->st), "synchronize");
    return FKMC_OK;
}

SiteArgs site_args(const kmc_batch* b)
{
    SiteArgs a{};
    a.vv = b->d_vv;
    a.btab = b->btab;
    a.field = b->field;
    a.n_vv = b->n_vv;
    a.e_self = b->e_self;
    a.gbound = b->grains_on ? b->gbound : nullptr;
    a.g_elec = b->elec_on ? b->d_elec_g : nullptr;
    return a;
}

// Rate tables of boundary hops: barriers raised by the grains' barrier, the
// mixed form quantised against the bulk table's k32max (same F).
int grain_tables(kmc_batch* b, int r)
{
    RepDesc& D = b->desc[r];
    if (!b->grains_on) {
        for (int i = 0; i < 6; ++i) {
            D.k64g[i] = D.k64[i];
            D.qg[i] = D.q[i];
        }
        return FKMC_OK;
    }
    kmc_barrier_table t = b->tables[r];
    t.Ea_O_eV += b->grains.barrier_eV;
    t.Ea_H_eV += b->grains.barrier_eV;
    float k32g[6], kmax = 0.0f;
    uint64_t qtmp[6];
    int32_t F;
    int rc = rate_table_impl(&t, b->T[r], b->Ez[r], b->a_ang[r], b->cap, D.k64g, k32g, qtmp, &F);
    if (rc) return rc;
    for (int i = 0; i < 6; ++i) kmax = std::max(kmax, (float)D.k64[i]);
    for (int i = 0; i < 6; ++i) D.qg[i] = (uint64_t)std::llrint(std::ldexp((double)k32g[i] / (double)kmax, D.F));
    return FKMC_OK;
}

int rebuild_field(kmc_batch* b)
{
    const SiteArgs a = site_args(b);
    CK(launch_site_field(b->d_desc, b->n, b->recs, b->counts, b->nfrag_total, b->cap, b->nsite_total, b->fe, b->d_bo,
                         b->n_bo, a, b->st),
       "energy field");
    if (b->elec_on) CK(elec_add(b->field, b->elec_u, b->nsite_total, b->st), "energy field");
    b->field_valid = true;
    return FKMC_OK;
}

void drop_window_graph(kmc_batch* b);

// the Boltzmann tables must cover electrostatic energies up to |u| = um
int elec_cover(kmc_batch* b, int64_t um)
{
    if (um <= b->elec_umax) return FKMC_OK;
    b->elec_umax = 2 * um + 1024;
    if (!b->rates_set) return FKMC_OK;  // kmc_set_barriers builds the tables
    const double* before = b->btab;
    int rc = build_btab(b);
    if (rc) return rc;
    rc = upload_desc(b);
    if (rc) return rc;
    if (b->btab != before) drop_window_graph(b);
    return FKMC_OK;
}

// V-cycles of the next automatic refresh
static int refresh_cycles(const kmc_batch* b)
{
    return b->phi_prev_valid && b->elec.warm_cycles > 0 ? b->elec.warm_cycles : b->elec.cycles;
}

// kernels of one refresh: per replica the solve (deposit, right-hand side,
// V-cycles, mean) and the update
uint64_t elec_launches(const kmc_batch* b)
{
    uint64_t k = 0;
    for (int r = 0; r < b->n; ++r) {
        const MgPlan p = mg_plan(b->desc[r].L[0], b->desc[r].L[1], b->desc[r].L[2]);
        k += 2 + (uint64_t)refresh_cycles(b) * mg_cycle_kernels(p) + 3 + 1;
    }
    return k;
}

// Potential of every replica's vacancy charges (multigrid), then u and the
// energy field moved to it; the Boltzmann tables grow if the bound does.
int elec_refresh(kmc_batch* b)
{
    CK(cudaMemsetAsync(b->d_umax, 0, sizeof(unsigned), b->st), "memset");
    const int cycles = refresh_cycles(b);
    const bool warm = b->phi_prev_valid, with_field = b->field_valid;
    if (!b->cap_st) CK(cudaStreamCreateWithFlags(&b->cap_st, cudaStreamNonBlocking), "stream");
    for (int r = 0; r < b->n; ++r) {
        // each replica's solve is one graph (some 40 launches per V-cycle); every
        // argument is fixed until the window graph is dropped, which drops these too
        cudaGraphExec_t exec = nullptr;
        for (auto& g : b->elec_graphs)
            if (g.r == r && g.cycles == cycles && g.warm == warm && g.field == with_field) exec = g.exec;
        if (!exec) {
            const RepDesc& D = b->desc[r];
            const MgPlan p = mg_plan(D.L[0], D.L[1], D.L[2]);
            const double scale = 1.602176634e-19 / (8.8541878128e-12 * b->elec.eps_r * b->a_ang[r] * 1e-10);
            double* prev = b->phi_prev + D.site_off / 3;
            cudaGraph_t graph = nullptr;
            CK(cudaStreamBeginCapture(b->cap_st, cudaStreamCaptureModeThreadLocal), "graph capture");
            cudaError_t le = elec_solve(D, b->recs, b->counts, b->cap, b->n_vac[r], b->elec.q_vac, scale, cycles, p,
                                        b->mgb, nullptr, warm ? prev : nullptr, prev, b->cap_st);
            if (le == cudaSuccess)
                le = elec_update(D, b->mgb.phi, b->elec.q_vac, b->elec_u, with_field ? b->field : nullptr, b->d_umax,
                                 b->cap_st);
            cudaError_t ce = cudaStreamEndCapture(b->cap_st, &graph);
            if (le != cudaSuccess) return cuda_fail(le, "potential solve capture");
            if (ce != cudaSuccess) return cuda_fail(ce, "potential solve capture");
            cudaError_t ie = cudaGraphInstantiate(&exec, graph, 0);
            cudaGraphDestroy(graph);
            if (ie != cudaSuccess) return cuda_fail(ie, "graph instantiate");
            b->elec_graphs.push_back({r, cycles, warm, with_field, exec});
        }
        CK(cudaGraphLaunch(exec, b->st), "graph launch");
    }
    unsigned um = 0;
    CK(cudaMemcpyAsync(&um, b->d_umax, sizeof um, cudaMemcpyDeviceToHost, b->st), "copy");
    CK(cudaStreamSynchronize(b->st), "synchronize");
    b->elec_age = 0;
    b->phi_prev_valid = true;
    return elec_cover(b, (int64_t)um);
}

// simulated time of the null-event form of replica r (s): its clock counts in 1/k32max
double null_time(const kmc_batch* b, int r)
{
    float kmax = 0.0f;
    for (int i = 0; i < 6; ++i) kmax = std::max(kmax, (float)b->desc[r].k64[i]);
    return kmax > 0.0f ? b->theta_host[r] / (double)kmax : 0.0;
}

void drop_window_graph(kmc_batch* b)
{
    if (b->window_exec) cudaGraphExecDestroy(b->window_exec);
    b->window_exec = nullptr;
    for (auto& g : b->elec_graphs) cudaGraphExecDestroy(g.exec);
    b->elec_graphs.clear();
}

}  // namespace

extern "C" {

const char* kmc_last_error(void) { return g_err.c_str(); }

void kmc_default_opts(kmc_opts* o)
{
    if (!o) return;
    std::memset(o, 0, sizeof *o);
    o->edge = 4;
    o->precision = FKMC_PLAIN;
    o->n_tau = 1.0;
    o->cluster_top = -1;
}

int32_t kmc_partition_count(int32_t L, int32_t edge)
{
    if (L < 1 || edge < 1) return 0;
    return partition_count(L, edge);
}

void kmc_neighbour_table(int32_t out[168])
{
    NbEntry tab[3][8];
    build_nb_table(tab);
    for (int t = 0; t < 3; ++t)
        for (int n = 0; n < 8; ++n) {
            int32_t* o = out + (t * 8 + n) * 7;
            o[0] = tab[t][n].t2;
            for (int k = 0; k < 3; ++k) {
                o[1 + k] = tab[t][n].dc[k];
                o[4 + k] = tab[t][n].d[k];
            }
        }
}

int kmc_rate_table(const kmc_barrier_table* t, double T_K, double field_z_Vpm, double a_angstrom,
                   int32_t cap_v, double k64[6], float k32[6], uint64_t q[6], int32_t* F)
{
    if (!k64 || !k32 || !q || !F) return fail(FKMC_EINVAL, "null output");
    return rate_table_impl(t, T_K, field_z_Vpm, a_angstrom, cap_v, k64, k32, q, F);
}

int kmc_create_batch(int32_t n, const kmc_cells* cells, const kmc_composition* comp, uint64_t seed,
                     const kmc_opts* opts_in, kmc_batch** out)
{
    if (!out) return fail(FKMC_EINVAL, "out is NULL");
    *out = nullptr;
    if (n < 1 || !cells || !comp) return fail(FKMC_EINVAL, "need n >= 1 replicas with cells and composition");
    kmc_opts o;
    kmc_default_opts(&o);
    if (opts_in) o = *opts_in;
    if (o.edge <= 0) o.edge = 4;
    if (!(o.n_tau > 0.0) || !(o.n_tau <= 64.0)) return fail(FKMC_EINVAL, "n_tau must be in (0, 64]");
    if (o.precision != FKMC_PLAIN && o.precision != FKMC_MIXED) return fail(FKMC_EINVAL, "bad precision");
    if (o.cap_v != 0 && (o.cap_v < 8 || o.cap_v > 256 || o.cap_v % 8))
        return fail(FKMC_EINVAL, "cap_v must be 0 or a multiple of 8 in [8, 256]");
    if (o.schedule < 0 || o.schedule > 2) return fail(FKMC_EINVAL, "schedule must be 0, 1 or 2");
    if (o.small_pass < -1 || o.small_pass > 2) return fail(FKMC_EINVAL, "small_pass must be -1, 0, 1 or 2");
    if (o.lane_form < 0 || o.lane_form > 2) return fail(FKMC_EINVAL, "lane_form must be 0, 1 or 2");
    if (o.cluster_ctas < -1 || o.cluster_ctas == 1 || o.cluster_ctas > CLUSTER_MAX_CTAS)
        return fail(FKMC_EINVAL, "cluster_ctas must be -1, 0 or 2..16");
    if (o.test_stuck_wait_us < 0 || o.test_stuck_wait_us > 2000000)
        return fail(FKMC_EINVAL, "test_stuck_wait_us must be in [0, 2e6]");

    kmc_batch* b = new kmc_batch();
    b->n = n;
    b->opts = o;
    b->st = (cudaStream_t)o.stream;
    b->desc.resize(n);
    b->n_vac.resize(n);
    b->n_H.resize(n);
    b->n_fe.assign(n, 0);
    b->T.assign(n, 0.0);
    b->theta_host.assign(n, 0.0);
    b->b_bits.resize(n);
    b->a_ang.resize(n);
    b->stats_host.assign(2 * (size_t)n, 0ull);
    double worst_mean = 0.0;
    for (int r = 0; r < n; ++r) {
        const kmc_cells& c = cells[r];
        const int L[3] = {c.nx, c.ny, c.nz};
        RepDesc& D = b->desc[r];
        std::memset(&D, 0, sizeof D);
        for (int d = 0; d < 3; ++d) {
            if (L[d] < 1 || L[d] > 65535) {
                delete b;
                return fail(FKMC_EINVAL, "cells per dimension must be in [1, 65535]");
            }
            D.L[d] = L[d];
            D.nf[d] = o.nfrag[d] > 0 ? o.nfrag[d] : partition_count(L[d], o.edge);
            if (!partition_ok(L[d], D.nf[d])) {
                delete b;
                return fail(FKMC_EINVAL, "fragments per dimension must be 1, or even with every edge >= 2");
            }
            D.base[d] = L[d] / D.nf[d];
            D.rem[d] = L[d] % D.nf[d];
        }
        if (!(c.a_angstrom > 0.0)) {
            delete b;
            return fail(FKMC_EINVAL, "lattice constant must be > 0");
        }
        D.nsite = 3 * (int64_t)L[0] * L[1] * L[2];
        if (comp[r].n_vac < 0 || comp[r].n_H < 0 || comp[r].n_vac + comp[r].n_H > D.nsite ||
            comp[r].n_vac > 0xffffffffll) {
            delete b;
            return fail(FKMC_EINVAL, "composition does not fit the lattice");
        }
        if (comp[r].n_Fe < 0 || comp[r].n_Fe > (int64_t)L[0] * L[1] * L[2]) {
            delete b;
            return fail(FKMC_EINVAL, "dopant count must be in [0, nx ny nz]");
        }
        b->n_vac[r] = comp[r].n_vac;
        b->n_H[r] = comp[r].n_H;
        b->n_fe[r] = comp[r].n_Fe;
        b->a_ang[r] = c.a_angstrom;
        D.replica = (uint32_t)r;
        D.seed = seed;
        D.row_words = (int32_t)(((L[0] + 63) / 64) * 4);  // 16 sites per word, rows padded to 16 bytes
        D.items = ((D.nf[0] + 1) / 2) * ((D.nf[1] + 1) / 2) * ((D.nf[2] + 1) / 2);
        D.items_off = b->total_items;
        b->total_items += D.items;
        const int64_t nfrag = (int64_t)D.nf[0] * D.nf[1] * D.nf[2];
        D.frag_base = b->nfrag_total;
        b->nfrag_total += nfrag;
        D.occ_word_off = b->occ_words;
        b->occ_words += 3 * (int64_t)L[2] * L[1] * D.row_words;
        D.site_off = b->nsite_total;
        b->nsite_total += D.nsite;
        int bb = 1;
        while (((int64_t)1 << (2 * bb)) < D.nsite) ++bb;
        b->b_bits[r] = bb;
        worst_mean = std::max(worst_mean, (double)comp[r].n_vac / (double)nfrag);
    }
    if (o.cap_v == 0) {
        int cap = (int)std::ceil(worst_mean + 10.0 * std::sqrt(worst_mean + 1.0) + 8.0);
        cap = ((cap + 7) / 8) * 8;
        b->cap = std::min(256, std::max(8, cap));
    } else {
        b->cap = o.cap_v;
    }
    b->opts.cap_v = b->cap;
    if (o.cluster_top >= 0) {
        b->cluster_top = o.cluster_top;
    } else {  // auto: the largest replicas take an extra SM each, about one SM in eight
        int dev = 0, sms = 0;
        if (cudaGetDevice(&dev) == cudaSuccess &&
            cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) == cudaSuccess)
            b->cluster_top = sms / 8;
        else
            b->cluster_top = 0;
    }

    b->occ = (uint32_t*)b->dalloc(sizeof(uint32_t) * b->occ_words);
    b->recs = (VacRec*)b->dalloc(sizeof(VacRec) * b->nfrag_total * b->cap);
    b->counts = (int32_t*)b->dalloc(sizeof(int32_t) * b->nfrag_total);
    if (o.tracer) b->tracer = (int32_t*)b->dalloc(sizeof(int32_t) * 3 * b->nsite_total);
    b->d_desc = (RepDesc*)b->dalloc(sizeof(RepDesc) * n);
    b->stats = (unsigned long long*)b->dalloc(sizeof(unsigned long long) * 2 * n);
    b->status = (uint32_t*)b->dalloc(sizeof(uint32_t));
    b->scratch = (unsigned long long*)b->dalloc(sizeof(unsigned long long) * 8);
    b->scratch_all = (unsigned long long*)b->dalloc(sizeof(unsigned long long) * 7 * n);
    b->d_reps = (int32_t*)b->dalloc(sizeof(int32_t) * n);
    b->d_plans = (ClusterPlan*)b->dalloc(sizeof(ClusterPlan) * n);
    b->rcache.tot = (unsigned long long*)b->dalloc(sizeof(unsigned long long) * std::max<int64_t>(b->nfrag_total, 1));
    b->rcache.dirty = (uint8_t*)b->dalloc((size_t)std::max<int64_t>(b->nfrag_total, 1));
    b->rcache.valid = (uint8_t*)b->dalloc((size_t)n);
    b->d_nvac = (int64_t*)b->dalloc(sizeof(int64_t) * n);
    b->wctl = (unsigned long long*)b->dalloc(sizeof(unsigned long long) * 2);
    b->perms = (uint32_t*)b->dalloc(sizeof(uint32_t) * n);
    b->act = (ActEntry*)b->dalloc(sizeof(ActEntry) * 3 * std::max<int64_t>(b->total_items, 1));
    b->act_count = (int32_t*)b->dalloc(sizeof(int32_t) * ACT_COUNTERS);
    b->cls = (uint8_t*)b->dalloc((size_t)std::max<int64_t>(b->total_items, 1));
    b->ncell_total = b->nsite_total / 3;
    bool any_fe = false;
    for (int r = 0; r < n; ++r) any_fe = any_fe || b->n_fe[r] > 0;
    if (any_fe) {
        b->fe = (uint8_t*)b->dalloc((size_t)b->ncell_total);
        if (!b->fe) {
            b->release();
            delete b;
            return fail(FKMC_ENOMEM, "device allocation failed");
        }
    }
    if (!b->occ || !b->recs || !b->counts || (o.tracer && !b->tracer) || !b->d_desc || !b->stats ||
        !b->status || !b->scratch || !b->scratch_all || !b->d_reps || !b->d_plans || !b->rcache.tot ||
        !b->rcache.dirty || !b->rcache.valid || !b->d_nvac || !b->wctl ||
        !b->perms ||
        !b->act || !b->act_count || !b->cls) {
        b->release();
        delete b;
        return fail(FKMC_ENOMEM, "device allocation failed");
    }
    int rc = FKMC_OK;
    auto step = [&](cudaError_t e, const char* what) {
        if (rc == FKMC_OK && e != cudaSuccess) rc = cuda_fail(e, what);
    };
    build_nb_table(b->nbt.e);
    step(upload_neighbours(&b->nbt.e[0][0]), "neighbour table upload");
    step(null_upload_neighbours(&b->nbt.e[0][0]), "neighbour table upload");
    step(phase_prepare(b->cap), "kernel attributes");
    step(run_pass_blocks(b->opts.precision, b->cap, false, false, &b->run_blocks), "occupancy query");
    step(resident_prepare(), "kernel attributes");
    step(cluster_prepare(), "kernel attributes");
    step(cudaEventCreateWithFlags(&b->fork, cudaEventDisableTiming), "event");
    step(cudaEventCreate(&b->ev0), "event");
    step(cudaEventCreate(&b->ev1), "event");
    step(cudaMemsetAsync(b->occ, 0, sizeof(uint32_t) * b->occ_words, b->st), "memset");
    step(cudaMemsetAsync(b->counts, 0, sizeof(int32_t) * b->nfrag_total, b->st), "memset");
    if (o.tracer) step(cudaMemsetAsync(b->tracer, 0, sizeof(int32_t) * 3 * b->nsite_total, b->st), "memset");
    step(cudaMemsetAsync(b->stats, 0, sizeof(unsigned long long) * 2 * n, b->st), "memset");
    step(cudaMemsetAsync(b->rcache.valid, 0, (size_t)n, b->st), "memset");
    step(cudaMemsetAsync(b->status, 0, sizeof(uint32_t), b->st), "memset");
    for (int r = 0; r < n && rc == FKMC_OK; ++r)
        step(launch_init(b->desc[r], b->b_bits[r], b->n_vac[r], b->n_vac[r] + b->n_H[r], b->occ, b->recs,
                         b->counts, b->cap, b->status, b->st),
             "init kernel");
    if (b->fe) {
        step(cudaMemsetAsync(b->fe, 0, (size_t)b->ncell_total, b->st), "memset");
        for (int r = 0; r < n && rc == FKMC_OK; ++r) {
            int bb = 1;
            while (((int64_t)1 << (2 * bb)) < b->desc[r].nsite / 3) ++bb;
            step(launch_init_dopants(b->desc[r], bb, b->n_fe[r], b->fe, b->st), "dopant kernel");
        }
    }
    if (rc == FKMC_OK) rc = upload_desc(b);
    if (rc == FKMC_OK) rc = check_status(b);
    if (rc != FKMC_OK) {
        std::string keep = g_err;
        b->release();
        delete b;
        g_err = keep;
        return rc;
    }
    *out = b;
    return FKMC_OK;
}

int kmc_create_lattice(const kmc_cells* cells, const kmc_composition* comp, uint64_t seed,
                       const kmc_opts* opts, kmc_batch** out)
{
    return kmc_create_batch(1, cells, comp, seed, opts, out);
}

int kmc_set_barriers(kmc_batch* b, const kmc_barrier_table* tables, const double* T_K,
                     const double* field_z_Vpm)
{
    if (!b || !tables || !T_K) return fail(FKMC_EINVAL, "null argument");
    std::vector<RepDesc> nd = b->desc;
    for (int r = 0; r < b->n; ++r) {
        RepDesc& D = nd[r];
        float k32[6];
        int32_t F;
        const double Ez = field_z_Vpm ? field_z_Vpm[r] : 0.0;
        int rc = rate_table_impl(&tables[r], T_K[r], Ez, b->a_ang[r], b->cap, D.k64, k32, D.q, &F);
        if (rc) return rc;
        double kmax = 0.0;
        float kmax32 = 0.0f;
        for (int i = 0; i < 6; ++i) {
            if ((i < 3 || b->n_H[r] > 0) && D.k64[i] > kmax) kmax = D.k64[i];
            kmax32 = std::max(kmax32, k32[i]);
        }
        D.F = F;
        D.two_pow_F = std::ldexp(1.0, F);
        D.tau = b->opts.n_tau / (8.0 * kmax);
        D.theta_tau = D.tau * (double)kmax32;
    }
    b->desc = nd;
    b->tables.assign(tables, tables + b->n);
    b->Ez.assign(b->n, 0.0);
    for (int r = 0; r < b->n; ++r) {
        b->T[r] = T_K[r];
        b->Ez[r] = field_z_Vpm ? field_z_Vpm[r] : 0.0;
    }
    int rc = FKMC_OK;
    for (int r = 0; r < b->n && rc == FKMC_OK; ++r) rc = grain_tables(b, r);
    if (rc) return rc;
    if (site_path(b)) {
        rc = build_btab(b);
        if (rc) return rc;
    }
    rc = plan_residency(b);
    if (rc) return rc;
    CK(cudaMemcpyAsync(b->d_nvac, b->n_vac.data(), sizeof(int64_t) * b->n, cudaMemcpyHostToDevice, b->st),
       "vacancy count upload");
    rc = upload_desc(b);
    if (rc) return rc;
    b->rates_set = true;
    return FKMC_OK;
}

int kmc_run(kmc_batch* b, uint64_t windows, kmc_run_stats* stats)
{
    NvtxRange nvtx_range("kmc_run");
    if (!b) return fail(FKMC_EINVAL, "null batch");
    if (!b->rates_set) return fail(FKMC_ESTATE, "kmc_set_barriers must come before kmc_run");
    std::vector<unsigned long long> before = b->stats_host;
    CK(cudaEventRecord(b->ev0, b->st), "event record");
    if (!b->rclass.empty() && windows > 0) {
        // replica-resident classes on forked streams, joined back: captured once
        // per window count into a graph (fork, one launch per class, join) and
        // replayed on the caller's stream
        if (!b->res_exec || b->res_exec_windows != windows) {
            if (b->res_exec) cudaGraphExecDestroy(b->res_exec);
            b->res_exec = nullptr;
            if (!b->cap_st) CK(cudaStreamCreateWithFlags(&b->cap_st, cudaStreamNonBlocking), "stream");
            cudaGraph_t graph = nullptr;
            CK(cudaStreamBeginCapture(b->cap_st, cudaStreamCaptureModeThreadLocal), "graph capture");
            cudaError_t le = cudaEventRecord(b->fork, b->cap_st);
            // largest classes first: their CTAs run longest and should take SMs first
            for (auto it = b->rclass.rbegin(); it != b->rclass.rend() && le == cudaSuccess; ++it) {
                auto& c = *it;
                le = cudaStreamWaitEvent(c.st, b->fork, 0);
                if (le == cudaSuccess && c.slabs)
                    le = launch_cluster(b->d_desc, b->d_plans + c.start, c.count, c.cluster, c.smem, windows, b->occ,
                                        b->recs, b->counts, b->tracer, b->stats, b->status, b->cap, b->nbt, b->rcache,
                                        c.st);
                else if (le == cudaSuccess)
                    le = launch_resident(b->d_desc, b->d_reps + c.start, c.count, b->d_nvac, c.smem, c.threads,
                                         c.cluster, windows, b->occ, b->recs, b->counts, b->tracer, b->stats,
                                         b->status, b->cap, b->nbt, (uint32_t)b->opts.test_stuck_wait_us, b->rcache,
                                         c.st);
                if (le == cudaSuccess) le = cudaEventRecord(c.done, c.st);
                if (le == cudaSuccess) le = cudaStreamWaitEvent(b->cap_st, c.done, 0);
            }
            cudaError_t ce = cudaStreamEndCapture(b->cap_st, &graph);
            if (le != cudaSuccess) return cuda_fail(le, "resident capture");
            if (ce != cudaSuccess) return cuda_fail(ce, "resident capture");
            cudaError_t ie = cudaGraphInstantiate(&b->res_exec, graph, 0);
            cudaGraphDestroy(graph);
            if (ie != cudaSuccess) {
                b->res_exec = nullptr;
                return cuda_fail(ie, "graph instantiate");
            }
            b->res_exec_windows = windows;
        }
        if (!b->res_st) {
            CK(cudaStreamCreateWithFlags(&b->res_st, cudaStreamNonBlocking), "stream");
            CK(cudaEventCreateWithFlags(&b->res_fork, cudaEventDisableTiming), "event");
            CK(cudaEventCreateWithFlags(&b->res_join, cudaEventDisableTiming), "event");
        }
        CK(cudaEventRecord(b->res_fork, b->st), "event record");
        CK(cudaStreamWaitEvent(b->res_st, b->res_fork, 0), "stream wait");
        CK(cudaGraphLaunch(b->res_exec, b->res_st), "graph launch");
        CK(cudaEventRecord(b->res_join, b->res_st), "event record");
    }
    uint64_t extra_launches = 0;
    if (site_path(b) && !b->field_valid) {
        int rc0 = rebuild_field(b);
        if (rc0) return rc0;
        extra_launches = (b->n_vv > 0) + (b->n_bo > 0);
    }
    // capture one window (set-up + 8 x (screen, run)); every argument is fixed until
    // the tables are rebuilt, which drops the graph
    auto ensure_graph = [&]() -> int {
        if (b->window_exec) return FKMC_OK;
        if (!b->cap_st) CK(cudaStreamCreateWithFlags(&b->cap_st, cudaStreamNonBlocking), "stream");
        cudaGraph_t graph = nullptr;
        int small_blocks = 1;
        const bool split = window_split(site_path(b), b->total_items, b->opts.small_pass);
        const int lane = window_lane(b->opts.precision, b->opts.small_pass, b->opts.lane_form, b->total_items);
        if (split) CK(small_pass_blocks(b->opts.precision, b->grains_on, lane, &small_blocks), "occupancy query");
        if (!b->side_st) {
            CK(cudaStreamCreateWithFlags(&b->side_st, cudaStreamNonBlocking), "stream");
            CK(cudaEventCreateWithFlags(&b->side_fork, cudaEventDisableTiming), "event");
            CK(cudaEventCreateWithFlags(&b->side_join, cudaEventDisableTiming), "event");
        }
        CK(cudaStreamBeginCapture(b->cap_st, cudaStreamCaptureModeThreadLocal), "graph capture");
        SiteArgs wa = site_args(b);
        if (!site_path(b)) wa.field = nullptr;  // the table-rate run pass
        cudaError_t le = launch_window(b->opts.precision, b->d_desc, b->n, b->total_items, b->wctl, b->perms, b->act,
                                       b->act_count, b->cls, b->occ, b->recs, b->counts, b->tracer, b->stats, b->status, b->cap,
                                       b->run_blocks, small_blocks, split, lane, wa, b->cap_st, b->side_st,
                                       b->side_fork, b->side_join);
        cudaError_t ce = cudaStreamEndCapture(b->cap_st, &graph);
        if (le != cudaSuccess) return cuda_fail(le, "window capture");
        if (ce != cudaSuccess) return cuda_fail(ce, "window capture");
        cudaError_t ie = cudaGraphInstantiate(&b->window_exec, graph, 0);
        cudaGraphDestroy(graph);
        if (ie != cudaSuccess) {
            b->window_exec = nullptr;
            return cuda_fail(ie, "graph instantiate");
        }
        return FKMC_OK;
    };
    if (b->any_global && windows > 0) {
        CK(cudaMemsetAsync(b->wctl, 0, sizeof(unsigned long long) * 2, b->st), "memset");
        const uint64_t every = b->elec_on ? (uint64_t)b->elec.refresh_windows : 0;
        for (uint64_t wk = 0; wk < windows; ++wk) {
            if (every > 0 && b->elec_age >= every) {  // the potential follows the vacancies
                int rc1 = elec_refresh(b);
                if (rc1) return rc1;
                extra_launches += elec_launches(b);
            }
            int rc2 = ensure_graph();
            if (rc2) return rc2;
            CK(cudaGraphLaunch(b->window_exec, b->st), "graph launch");
            ++b->elec_age;
        }
    }
    if (!b->rclass.empty() && windows > 0) CK(cudaStreamWaitEvent(b->st, b->res_join, 0), "stream wait");
    CK(cudaEventRecord(b->ev1, b->st), "event record");
    for (int r = 0; r < b->n; ++r) b->desc[r].window += windows;
    int rc = upload_desc(b);
    if (rc) return rc;
    CK(cudaMemcpyAsync(b->stats_host.data(), b->stats, sizeof(unsigned long long) * 2 * b->n,
                       cudaMemcpyDeviceToHost, b->st),
       "stats copy");
    rc = check_status(b);
    if (stats) {
        std::memset(stats, 0, sizeof *stats);
        for (int r = 0; r < b->n; ++r) {
            stats->hops += b->stats_host[2 * r] - before[2 * r];
            stats->handoffs += b->stats_host[2 * r + 1] - before[2 * r + 1];
        }
        stats->windows = windows;
        stats->launches =
            (windows > 0 ? b->rclass.size() : 0) +
            (b->any_global ? window_launches(b) * windows : 0) +
            extra_launches;
        float ms = 0.f;
        cudaEventElapsedTime(&ms, b->ev0, b->ev1);
        stats->gpu_ms = ms;
    }
    return rc;
}

int kmc_run_null(kmc_batch* b, uint64_t steps, int64_t n_frg, kmc_run_stats* stats)
{
    NvtxRange nvtx_range("kmc_run_null");
    if (!b) return fail(FKMC_EINVAL, "null batch");
    if (!b->rates_set) return fail(FKMC_ESTATE, "kmc_set_barriers must come before kmc_run_null");
    if (site_path(b)) return fail(FKMC_EINVAL, "the null-event form has no site energies or electrostatics");
    if (n_frg < 1) return fail(FKMC_EINVAL, "n_frg must be >= 1");
    if (steps > 0xFFFFFFF0ull) return fail(FKMC_EINVAL, "at most 2^32 - 16 steps per call");
    // per-replica tables and offsets
    int64_t total_vac = 0, total_picks = 0;
    for (int r = 0; r < b->n; ++r) {
        RepDesc& D = b->desc[r];
        float k32[6], kmax = 0.0f;
        for (int i = 0; i < 6; ++i) {
            k32[i] = (float)D.k64[i];
            kmax = std::max(kmax, k32[i]);
        }
        const int64_t nv = b->n_vac[r];
        const int F = 63 - ceil_log2(8 * std::max<int64_t>(nv, 1));
        for (int i = 0; i < 6; ++i) D.qn[i] = (uint64_t)std::llrint(std::ldexp((double)k32[i] / (double)kmax, F));
        for (int i = 0; i < 6; ++i)
            D.qng[i] = b->grains_on ? (uint64_t)std::llrint(std::ldexp((double)(float)D.k64g[i] / (double)kmax, F))
                                    : D.qn[i];
        D.two_pow_Fn = std::ldexp(1.0, F);
        D.vac_off = total_vac;
        D.null_nv = nv;
        D.null_nfrg = std::min<int64_t>(n_frg, nv);
        D.pick_off = total_picks;
        total_vac += nv;
        total_picks += D.null_nfrg;
    }
    if (total_vac > b->vac_cap) {
        b->dfree(b->vac);
        b->vac = (VacRec*)b->dalloc(sizeof(VacRec) * total_vac);
        b->vac_cap = b->vac ? total_vac : 0;
        if (!b->vac) return fail(FKMC_ENOMEM, "device allocation failed (null-event vacancies)");
        if (b->null_exec) cudaGraphExecDestroy(b->null_exec);
        b->null_exec = nullptr;
    }
    if (!b->claims) {
        b->claims = (unsigned long long*)b->dalloc(sizeof(unsigned long long) * b->nsite_total);
        b->nacc = (unsigned long long*)b->dalloc(sizeof(unsigned long long) * 3 * b->n);
        b->theta = (double*)b->dalloc(sizeof(double) * b->n);
        b->nE = (double*)b->dalloc(sizeof(double) * b->n);
        b->nctl = (unsigned long long*)b->dalloc(sizeof(unsigned long long) * 3);
        if (!b->claims || !b->nacc || !b->theta || !b->nE || !b->nctl)
            return fail(FKMC_ENOMEM, "device allocation failed (null-event buffers)");
        CK(cudaMemcpyAsync(b->theta, b->theta_host.data(), sizeof(double) * b->n, cudaMemcpyHostToDevice, b->st),
           "clock upload");
    }
    if (total_picks > b->props_cap) {
        if (b->null_exec) cudaGraphExecDestroy(b->null_exec);
        b->null_exec = nullptr;
        b->dfree(b->props);
        b->props = (NullProp*)b->dalloc(sizeof(NullProp) * total_picks);
        if (!b->props) {
            b->props_cap = 0;
            return fail(FKMC_ENOMEM, "device allocation failed (null-event picks)");
        }
        b->props_cap = total_picks;
    }
    int rc = upload_desc(b);
    if (rc) return rc;
    std::vector<unsigned long long> before = b->stats_host;
    CK(cudaEventRecord(b->ev0, b->st), "event record");
    uint64_t launches = 0;
    CK(cudaMemsetAsync(b->claims, 0xFF, sizeof(unsigned long long) * b->nsite_total, b->st), "memset");
    CK(cudaMemsetAsync(b->nacc, 0, sizeof(unsigned long long) * 3 * b->n, b->st), "memset");
    CK(cudaMemsetAsync(b->nctl, 0, sizeof(unsigned long long) * 3, b->st), "memset");
    CK(launch_null_gather(b->d_desc, b->n, b->recs, b->counts, b->nfrag_total, b->cap, b->vac, b->status, b->st),
       "null gather");
    ++launches;
    if (steps > 0 && total_vac > 0) {
        if (!b->null_exec || b->null_exec_picks != total_picks || b->null_exec_vac != total_vac ||
            b->null_exec_grains != b->grains_on) {
            if (b->null_exec) cudaGraphExecDestroy(b->null_exec);
            b->null_exec = nullptr;
            if (!b->cap_st) CK(cudaStreamCreateWithFlags(&b->cap_st, cudaStreamNonBlocking), "stream");
            cudaGraph_t graph = nullptr;
            CK(cudaStreamBeginCapture(b->cap_st, cudaStreamCaptureModeThreadLocal), "graph capture");
            cudaError_t le = launch_null_step(b->d_desc, b->n, total_vac, total_picks, b->vac, b->occ,
                                              b->grains_on ? b->gbound : nullptr, b->nacc, b->props, b->claims,
                                              b->tracer, b->theta, b->nE, b->stats, b->nctl, b->cap_st);
            cudaError_t ce = cudaStreamEndCapture(b->cap_st, &graph);
            if (le != cudaSuccess) return cuda_fail(le, "null step capture");
            if (ce != cudaSuccess) return cuda_fail(ce, "null step capture");
            cudaError_t ie = cudaGraphInstantiate(&b->null_exec, graph, 0);
            cudaGraphDestroy(graph);
            if (ie != cudaSuccess) {
                b->null_exec = nullptr;
                return cuda_fail(ie, "graph instantiate");
            }
            b->null_exec_picks = total_picks;
            b->null_exec_vac = total_vac;
            b->null_exec_grains = b->grains_on;
        }
        for (uint64_t k = 0; k < steps; ++k) CK(cudaGraphLaunch(b->null_exec, b->st), "graph launch");
        launches += 3 * steps;
    }
    CK(launch_null_scatter(b->d_desc, b->n, total_vac, b->vac, b->recs, b->counts, b->nfrag_total, b->cap, b->status,
                           b->st),
       "null scatter");
    ++launches;
    CK(cudaEventRecord(b->ev1, b->st), "event record");
    for (int r = 0; r < b->n; ++r) b->desc[r].null_step += steps;
    rc = upload_desc(b);
    if (rc) return rc;
    CK(cudaMemcpyAsync(b->stats_host.data(), b->stats, sizeof(unsigned long long) * 2 * b->n, cudaMemcpyDeviceToHost,
                       b->st),
       "stats copy");
    CK(cudaMemcpyAsync(b->theta_host.data(), b->theta, sizeof(double) * b->n, cudaMemcpyDeviceToHost, b->st),
       "clock copy");
    rc = check_status(b);
    b->field_valid = false;
    {
        const int rc_ = drop_resident_cache(b);
        if (rc_) return rc_;
    }
    if (stats) {
        std::memset(stats, 0, sizeof *stats);
        for (int r = 0; r < b->n; ++r) stats->hops += b->stats_host[2 * r] - before[2 * r];
        stats->windows = 0;
        stats->launches = launches;
        float ms = 0.f;
        cudaEventElapsedTime(&ms, b->ev0, b->ev1);
        stats->gpu_ms = ms;
    }
    return rc;
}

int kmc_read_moments(kmc_batch* b, int32_t r, int32_t species, int64_t out[7])
{
    if (!valid_replica(b, r) || !out) return fail(FKMC_EINVAL, "bad replica or output");
    if (species != FKMC_O && species != FKMC_H && species != FKMC_V) return fail(FKMC_EINVAL, "bad species");
    if (species != FKMC_V && !b->tracer) return fail(FKMC_ESTATE, "ion moments need tracer mode");
    CK(launch_moments(b->desc[r], species, b->occ, b->recs, b->counts, b->tracer, b->cap, b->scratch, b->st),
       "moments kernel");
    unsigned long long h[7];
    CK(cudaMemcpyAsync(h, b->scratch, sizeof h, cudaMemcpyDeviceToHost, b->st), "moments copy");
    CK(cudaStreamSynchronize(b->st), "synchronize");
    for (int k = 0; k < 7; ++k) out[k] = (int64_t)h[k];
    return FKMC_OK;
}

int kmc_read_moments_all(kmc_batch* b, int64_t* out, size_t n_out)
{
    if (!b || !out) return fail(FKMC_EINVAL, "null argument");
    if (n_out != 7 * (size_t)b->n) return fail(FKMC_EINVAL, "n_out must be 7 x replicas");
    int64_t max_frag = 0;
    for (const RepDesc& D : b->desc) max_frag = std::max<int64_t>(max_frag, (int64_t)D.nf[0] * D.nf[1] * D.nf[2]);
    CK(launch_moments_all(b->d_desc, b->n, b->recs, b->counts, max_frag, b->cap, b->scratch_all, b->st),
       "moments kernel");
    CK(cudaMemcpyAsync(out, b->scratch_all, sizeof(int64_t) * n_out, cudaMemcpyDeviceToHost, b->st),
       "moments copy");
    CK(cudaStreamSynchronize(b->st), "synchronize");
    return FKMC_OK;
}

int kmc_read_msd(kmc_batch* b, int32_t r, int32_t species, double msd_xyz[3], double mean_xyz[3],
                 double* t_s)
{
    int64_t m[7];
    int rc = kmc_read_moments(b, r, species, m);
    if (rc) return rc;
    const double h = 0.5 * b->a_ang[r] * 1e-10;
    const double n = m[0] > 0 ? (double)m[0] : 1.0;
    for (int k = 0; k < 3; ++k) {
        if (msd_xyz) msd_xyz[k] = (double)m[4 + k] / n * h * h;
        if (mean_xyz) mean_xyz[k] = (double)m[1 + k] / n * h;
    }
    if (t_s) *t_s = (double)b->desc[r].window * b->desc[r].tau + null_time(b, r);
    return FKMC_OK;
}

int kmc_read_D(kmc_batch* b, int32_t r, int32_t species, double D_xyz[3], double* D, double* D_xy,
               double v_drift[3])
{
    double msd[3], mean[3], t;
    int rc = kmc_read_msd(b, r, species, msd, mean, &t);
    if (rc) return rc;
    if (!(t > 0.0)) return fail(FKMC_ESTATE, "no simulated time yet");
    for (int k = 0; k < 3; ++k) {
        // the variance of the displacement along each axis: the drift is removed
        if (D_xyz) D_xyz[k] = (msd[k] - mean[k] * mean[k]) / (2.0 * t);
        if (v_drift) v_drift[k] = mean[k] / t;
    }
    if (D) *D = (msd[0] + msd[1] + msd[2]) / (6.0 * t);
    if (D_xy) *D_xy = (msd[0] + msd[1]) / (4.0 * t);
    return FKMC_OK;
}

int kmc_read_state(kmc_batch* b, int32_t r, uint8_t* host_occ, size_t n)
{
    if (!valid_replica(b, r) || !host_occ) return fail(FKMC_EINVAL, "bad replica or output");
    const RepDesc& D = b->desc[r];
    if ((int64_t)n != D.nsite) return fail(FKMC_EINVAL, "n must equal 3 nx ny nz");
    const int64_t words = 3 * (int64_t)D.L[2] * D.L[1] * D.row_words;
    std::vector<uint32_t> w(words);
    CK(cudaMemcpyAsync(w.data(), b->occ + D.occ_word_off, sizeof(uint32_t) * words, cudaMemcpyDeviceToHost,
                       b->st),
       "state copy");
    CK(cudaStreamSynchronize(b->st), "synchronize");
    int64_t s = 0;
    for (int t = 0; t < 3; ++t)
        for (int z = 0; z < D.L[2]; ++z)
            for (int y = 0; y < D.L[1]; ++y) {
                for (int x = 0; x < D.L[0]; ++x)
                    host_occ[s++] = (uint8_t)((w[occ_index(D.row_words, D.L[1], t, x, y, z)] >> ((x & 15) * 2)) & 3u);
            }
    return FKMC_OK;
}

int kmc_write_state(kmc_batch* b, int32_t r, const uint8_t* host_occ, size_t n)
{
    if (!valid_replica(b, r) || !host_occ) return fail(FKMC_EINVAL, "bad replica or input");
    const RepDesc& D = b->desc[r];
    if ((int64_t)n != D.nsite) return fail(FKMC_EINVAL, "n must equal 3 nx ny nz");
    const int64_t words = 3 * (int64_t)D.L[2] * D.L[1] * D.row_words;
    const int64_t nfrag = (int64_t)D.nf[0] * D.nf[1] * D.nf[2];
    std::vector<uint32_t> w(words, 0u);
    std::vector<int32_t> cnt(nfrag, 0);
    std::vector<VacRec> rec((size_t)nfrag * b->cap);
    int64_t s = 0, nv = 0, nh = 0;
    for (int t = 0; t < 3; ++t)
        for (int z = 0; z < D.L[2]; ++z)
            for (int y = 0; y < D.L[1]; ++y) {
                for (int x = 0; x < D.L[0]; ++x, ++s) {
                    const uint8_t c = host_occ[s];
                    if (c > 2) return fail(FKMC_EINVAL, "species codes must be 0, 1 or 2");
                    w[occ_index(D.row_words, D.L[1], t, x, y, z)] |= (uint32_t)c << ((x & 15) * 2);
                    if (c == FKMC_H) ++nh;
                    if (c != FKMC_V) continue;
                    int f[3];
                    const int cc[3] = {x, y, z};
                    for (int d = 0; d < 3; ++d) {
                        const int big = D.rem[d] * (D.base[d] + 1);
                        f[d] = cc[d] < big ? cc[d] / (D.base[d] + 1) : D.rem[d] + (cc[d] - big) / D.base[d];
                    }
                    const int64_t g = ((int64_t)f[2] * D.nf[1] + f[1]) * D.nf[0] + f[0];
                    if (cnt[g] >= b->cap) return fail(FKMC_EOVERFLOW, "a fragment would exceed cap_v vacancies");
                    VacRec& v = rec[g * b->cap + cnt[g]++];
                    v.key = ((uint64_t)t << 48) | ((uint64_t)z << 32) | ((uint64_t)y << 16) | (uint64_t)x;
                    v.d[0] = v.d[1] = v.d[2] = 0;
                    v.id = (uint32_t)nv++;
                }
            }
    CK(cudaMemcpyAsync(b->occ + D.occ_word_off, w.data(), sizeof(uint32_t) * words, cudaMemcpyHostToDevice,
                       b->st),
       "state upload");
    CK(cudaMemcpyAsync(b->counts + D.frag_base, cnt.data(), sizeof(int32_t) * nfrag, cudaMemcpyHostToDevice,
                       b->st),
       "count upload");
    CK(cudaMemcpyAsync(b->recs + D.frag_base * b->cap, rec.data(), sizeof(VacRec) * rec.size(),
                       cudaMemcpyHostToDevice, b->st),
       "record upload");
    if (b->tracer)
        CK(cudaMemsetAsync(b->tracer + 3 * D.site_off, 0, sizeof(int32_t) * 3 * D.nsite, b->st), "memset");
    CK(cudaStreamSynchronize(b->st), "synchronize");
    b->n_vac[r] = nv;
    b->n_H[r] = nh;
    b->field_valid = false;
    {
        const int rc_ = drop_resident_cache(b);
        if (rc_) return rc_;
    }
    b->elec_age = UINT64_MAX / 2;  // the potential is solved again at the next refresh point
    b->phi_prev_valid = false;  // and from zero: the vacancies may have moved anywhere
    drop_window_graph(b);       // the captured solves hold the vacancy count
    if (b->rates_set) {
        int rc = plan_residency(b);
        if (rc) return rc;
        CK(cudaMemcpyAsync(b->d_nvac, b->n_vac.data(), sizeof(int64_t) * b->n, cudaMemcpyHostToDevice, b->st),
           "vacancy count upload");
        rc = upload_desc(b);
        if (rc) return rc;
    }
    return FKMC_OK;
}

int kmc_read_records(kmc_batch* b, int32_t r, int64_t* rows, int64_t max_rows, int64_t* n_rows)
{
    if (!valid_replica(b, r) || (!rows && max_rows > 0)) return fail(FKMC_EINVAL, "bad replica or output");
    const RepDesc& D = b->desc[r];
    const int64_t nfrag = (int64_t)D.nf[0] * D.nf[1] * D.nf[2];
    std::vector<int32_t> cnt(nfrag);
    std::vector<VacRec> rec((size_t)nfrag * b->cap);
    CK(cudaMemcpyAsync(cnt.data(), b->counts + D.frag_base, sizeof(int32_t) * nfrag, cudaMemcpyDeviceToHost,
                       b->st),
       "count copy");
    CK(cudaMemcpyAsync(rec.data(), b->recs + D.frag_base * b->cap, sizeof(VacRec) * rec.size(),
                       cudaMemcpyDeviceToHost, b->st),
       "record copy");
    CK(cudaStreamSynchronize(b->st), "synchronize");
    int64_t k = 0, total = 0;
    for (int64_t f = 0; f < nfrag; ++f) {
        const int c = std::min(cnt[f], b->cap);
        total += c;
        std::vector<std::pair<int64_t, int>> lst;
        for (int m = 0; m < c; ++m) {
            const VacRec& v = rec[f * b->cap + m];
            const int64_t x = v.key & 0xffff, y = (v.key >> 16) & 0xffff, z = (v.key >> 32) & 0xffff,
                          t = (int64_t)(v.key >> 48);
            lst.push_back({((t * D.L[2] + z) * D.L[1] + y) * D.L[0] + x, m});
        }
        std::sort(lst.begin(), lst.end());
        for (auto& pr : lst) {
            if (k >= max_rows) break;
            const VacRec& v = rec[f * b->cap + pr.second];
            int64_t* o = rows + 6 * k++;
            o[0] = f;
            o[1] = pr.first;
            o[2] = v.d[0];
            o[3] = v.d[1];
            o[4] = v.d[2];
            o[5] = v.id;
        }
    }
    if (n_rows) *n_rows = total;
    return FKMC_OK;
}

int kmc_read_tracer(kmc_batch* b, int32_t r, int32_t* host_disp, size_t n_sites)
{
    if (!valid_replica(b, r) || !host_disp) return fail(FKMC_EINVAL, "bad replica or output");
    if (!b->tracer) return fail(FKMC_ESTATE, "tracer mode is off");
    const RepDesc& D = b->desc[r];
    if ((int64_t)n_sites != D.nsite) return fail(FKMC_EINVAL, "n_sites must equal 3 nx ny nz");
    CK(cudaMemcpyAsync(host_disp, b->tracer + 3 * D.site_off, sizeof(int32_t) * 3 * D.nsite,
                       cudaMemcpyDeviceToHost, b->st),
       "tracer copy");
    CK(cudaStreamSynchronize(b->st), "synchronize");
    return FKMC_OK;
}

}  // extern "C"

namespace {

// The state blob: a header, one row of counters per replica, then every
// mutable device array of the batch (each part starts on an 8-byte boundary).
constexpr uint64_t BLOB_MAGIC = 0x31415453434d4b46ull;  // "FKMCSTA1"
enum : uint32_t { BLOB_TRACER = 1u, BLOB_DOPANTS = 2u, BLOB_ELEC = 4u };
struct BlobHeader {
    uint64_t magic;
    uint32_t n, flags;
    uint64_t occ_words, nfrag_total, cap, nsite_total;
    uint64_t elec_age, phi_prev_valid;
};
struct BlobReplica {
    uint64_t window, null_step, hops, handoffs;
    double null_theta;
    int64_t n_vac, n_H;
};
static_assert(sizeof(BlobHeader) == 64 && sizeof(BlobReplica) == 56, "blob layout");

uint32_t blob_flags(const kmc_batch* b)
{
    return (b->tracer ? BLOB_TRACER : 0u) | (b->fe ? BLOB_DOPANTS : 0u) | (b->elec_on ? BLOB_ELEC : 0u);
}

struct BlobPart {
    void* dev;
    size_t bytes;
};

// the device arrays of the blob in order, and the header + rows size
size_t blob_parts(const kmc_batch* b, std::vector<BlobPart>* parts)
{
    const uint32_t f = blob_flags(b);
    parts->clear();
    parts->push_back({b->occ, sizeof(uint32_t) * b->occ_words});
    parts->push_back({b->recs, sizeof(VacRec) * b->nfrag_total * b->cap});
    parts->push_back({b->counts, sizeof(int32_t) * b->nfrag_total});
    if (f & BLOB_TRACER) parts->push_back({b->tracer, sizeof(int32_t) * 3 * b->nsite_total});
    if (f & BLOB_DOPANTS) parts->push_back({b->fe, (size_t)b->ncell_total});
    if (f & BLOB_ELEC) {
        parts->push_back({b->elec_u, sizeof(int32_t) * b->nsite_total});
        parts->push_back({b->phi_prev, sizeof(double) * b->ncell_total});
    }
    return sizeof(BlobHeader) + sizeof(BlobReplica) * (size_t)b->n;
}

size_t align8(size_t v) { return (v + 7) & ~(size_t)7; }

}  // namespace

extern "C" {

int kmc_state_bytes(kmc_batch* b, size_t* bytes)
{
    if (!b || !bytes) return fail(FKMC_EINVAL, "null argument");
    std::vector<BlobPart> parts;
    size_t total = blob_parts(b, &parts);
    for (const BlobPart& p : parts) total = align8(total) + p.bytes;
    *bytes = align8(total);
    return FKMC_OK;
}

int kmc_download_state(kmc_batch* b, void* host, size_t bytes)
{
    size_t need = 0;
    int rc = kmc_state_bytes(b, &need);
    if (rc) return rc;
    if (!host || bytes != need) return fail(FKMC_EINVAL, "buffer size must equal kmc_state_bytes");
    char* h = (char*)host;
    std::vector<BlobPart> parts;
    size_t off = blob_parts(b, &parts);
    BlobHeader hd{};
    hd.magic = BLOB_MAGIC;
    hd.n = (uint32_t)b->n;
    hd.flags = blob_flags(b);
    hd.occ_words = (uint64_t)b->occ_words;
    hd.nfrag_total = (uint64_t)b->nfrag_total;
    hd.cap = (uint64_t)b->cap;
    hd.nsite_total = (uint64_t)b->nsite_total;
    hd.elec_age = b->elec_age;
    hd.phi_prev_valid = b->phi_prev_valid ? 1u : 0u;
    std::memcpy(h, &hd, sizeof hd);
    for (int r = 0; r < b->n; ++r) {
        BlobReplica row{b->desc[r].window, b->desc[r].null_step, b->stats_host[2 * r], b->stats_host[2 * r + 1],
                        b->theta_host[r], b->n_vac[r], b->n_H[r]};
        std::memcpy(h + sizeof hd + sizeof row * r, &row, sizeof row);
    }
    for (const BlobPart& p : parts) {
        off = align8(off);
        CK(cudaMemcpyAsync(h + off, p.dev, p.bytes, cudaMemcpyDeviceToHost, b->st), "state copy");
        off += p.bytes;
    }
    CK(cudaStreamSynchronize(b->st), "synchronize");
    return FKMC_OK;
}

int kmc_upload_state(kmc_batch* b, const void* host, size_t bytes)
{
    size_t need = 0;
    int rc = kmc_state_bytes(b, &need);
    if (rc) return rc;
    if (!host || bytes != need) return fail(FKMC_EINVAL, "buffer size must equal kmc_state_bytes");
    const char* h = (const char*)host;
    BlobHeader hd;
    std::memcpy(&hd, h, sizeof hd);
    if (hd.magic != BLOB_MAGIC || hd.n != (uint32_t)b->n || hd.flags != blob_flags(b) ||
        hd.occ_words != (uint64_t)b->occ_words || hd.nfrag_total != (uint64_t)b->nfrag_total ||
        hd.cap != (uint64_t)b->cap || hd.nsite_total != (uint64_t)b->nsite_total)
        return fail(FKMC_EINVAL, "state blob of another batch shape (replicas, sizes, cap_v, tracer, dopants, "
                                 "electrostatics)");
    std::vector<BlobReplica> rows(b->n);
    for (int r = 0; r < b->n; ++r) {
        std::memcpy(&rows[r], h + sizeof hd + sizeof(BlobReplica) * r, sizeof(BlobReplica));
        if (rows[r].n_vac < 0 || rows[r].n_H < 0 || rows[r].n_vac + rows[r].n_H > b->desc[r].nsite)
            return fail(FKMC_EINVAL, "state blob: bad composition");
    }
    std::vector<BlobPart> parts;
    size_t off = blob_parts(b, &parts);
    for (const BlobPart& p : parts) {
        off = align8(off);
        CK(cudaMemcpyAsync(p.dev, h + off, p.bytes, cudaMemcpyHostToDevice, b->st), "state upload");
        off += p.bytes;
    }
    for (int r = 0; r < b->n; ++r) {
        b->desc[r].window = rows[r].window;
        b->desc[r].null_step = rows[r].null_step;
        b->stats_host[2 * r] = rows[r].hops;
        b->stats_host[2 * r + 1] = rows[r].handoffs;
        b->theta_host[r] = rows[r].null_theta;
        b->n_vac[r] = rows[r].n_vac;
        b->n_H[r] = rows[r].n_H;
    }
    CK(cudaMemcpyAsync(b->stats, b->stats_host.data(), sizeof(unsigned long long) * 2 * b->n, cudaMemcpyHostToDevice,
                       b->st),
       "counter upload");
    if (b->theta)
        CK(cudaMemcpyAsync(b->theta, b->theta_host.data(), sizeof(double) * b->n, cudaMemcpyHostToDevice, b->st),
           "clock upload");
    CK(cudaStreamSynchronize(b->st), "synchronize");
    b->field_valid = false;  // the site-energy field is rebuilt from the restored vacancies, dopants and u
    {
        const int rc_ = drop_resident_cache(b);
        if (rc_) return rc_;
    }
    if (blob_flags(b) & BLOB_ELEC) {
        b->elec_age = hd.elec_age;
        b->phi_prev_valid = hd.phi_prev_valid != 0;
    } else {
        b->elec_age = UINT64_MAX / 2;
        b->phi_prev_valid = false;
    }
    drop_window_graph(b);  // the captured solves hold the vacancy counts
    if (b->rates_set) {
        rc = plan_residency(b);
        if (rc) return rc;
        CK(cudaMemcpyAsync(b->d_nvac, b->n_vac.data(), sizeof(int64_t) * b->n, cudaMemcpyHostToDevice, b->st),
           "vacancy count upload");
    }
    return upload_desc(b);
}

int kmc_set_site_energy(kmc_batch* b, const kmc_site_energy* e)
{
    if (!b) return fail(FKMC_EINVAL, "null batch");
    if (!e || (e->n_vv == 0 && e->n_fe == 0)) {
        if (b->site_on) {
            b->site_on = false;
            b->n_vv = b->n_bo = b->e_self = 0;  // electrostatics may keep the site-energy pass
            b->e_bound = 0;
            b->field_valid = false;
            {
                const int rc_ = drop_resident_cache(b);
                if (rc_) return rc_;
            }
            drop_window_graph(b);
            CK(run_pass_blocks(site_path(b) ? FKMC_PLAIN : b->opts.precision, b->cap, site_path(b), b->grains_on,
                               &b->run_blocks),
               "occupancy query");
            if (b->rates_set) {
                int rc = plan_residency(b);
                if (rc) return rc;
                rc = upload_desc(b);
                if (rc) return rc;
            }
        }
        return FKMC_OK;
    }
    if (b->opts.precision != FKMC_PLAIN) return fail(FKMC_EINVAL, "site energies need the plain form");
    ShellTables sh;
    int rc0 = make_shells(e, &sh);
    if (rc0) return rc0;
    const int reach_all = sh.reach_all, reach_vv = sh.reach_vv;
    const std::vector<SiteOff>& vv = sh.vv;
    const std::vector<SiteOff>& bo = sh.bo;
    for (int r = 0; r < b->n; ++r)
        for (int d = 0; d < 3; ++d) {
            const RepDesc& D = b->desc[r];
            if (D.L[d] < 2 * reach_all + 1)
                return fail(FKMC_EINVAL, "a dimension is shorter than twice the interaction reach plus one cell");
            if (D.nf[d] > 1 && D.base[d] < 2 + reach_vv)
                return fail(FKMC_EINVAL, "fragment edges must be at least 2 + the V-V reach (cells)");
        }
    const int32_t eself = sh.e_self;

    if (!b->field) b->field = (int32_t*)b->dalloc(sizeof(int32_t) * b->nsite_total);
    if (!b->d_vv) b->d_vv = (SiteOff*)b->dalloc(sizeof(SiteOff) * 3 * SITE_MAX_VV);
    if (!b->d_bo) b->d_bo = (SiteOff*)b->dalloc(sizeof(SiteOff) * SITE_MAX_BO);
    if (!b->fe) {
        b->fe = (uint8_t*)b->dalloc((size_t)b->ncell_total);
        if (b->fe) CK(cudaMemsetAsync(b->fe, 0, (size_t)b->ncell_total, b->st), "memset");
    }
    if (!b->field || !b->d_vv || !b->d_bo || !b->fe) return fail(FKMC_ENOMEM, "device allocation failed");
    b->n_vv = sh.nvv;
    b->n_bo = (int)bo.size();
    b->e_self = eself;
    b->e_bound = sh.bound;
    CK(cudaMemcpyAsync(b->d_vv, vv.data(), sizeof(SiteOff) * vv.size(), cudaMemcpyHostToDevice, b->st),
       "table upload");
    if (!bo.empty())
        CK(cudaMemcpyAsync(b->d_bo, bo.data(), sizeof(SiteOff) * bo.size(), cudaMemcpyHostToDevice, b->st),
           "table upload");
    b->site_on = true;
    b->field_valid = false;
    {
        const int rc_ = drop_resident_cache(b);
        if (rc_) return rc_;
    }
    drop_window_graph(b);
    CK(run_pass_blocks(FKMC_PLAIN, b->cap, true, b->grains_on, &b->run_blocks), "occupancy query");
    if (b->rates_set) {
        int rc = build_btab(b);
        if (rc) return rc;
        rc = plan_residency(b);
        if (rc) return rc;
        rc = upload_desc(b);
        if (rc) return rc;
    }
    CK(cudaStreamSynchronize(b->st), "synchronize");
    return FKMC_OK;
}

int kmc_site_shells(const kmc_site_energy* e, int32_t t, int32_t* rows, int32_t max_rows, int32_t* n_rows)
{
    if (!e || t < 0 || t > 2 || (!rows && max_rows > 0)) return fail(FKMC_EINVAL, "bad argument");
    ShellTables sh;
    int rc = make_shells(e, &sh);
    if (rc) return rc;
    int k = 0;
    auto put = [&](const SiteOff& o) {
        if (k < max_rows) {
            int32_t* w = rows + 5 * k;
            w[0] = o.t2;
            for (int a = 0; a < 3; ++a) w[1 + a] = o.dc[a];
            w[4] = o.e;
        }
        ++k;
    };
    for (int i = 0; i < sh.nvv; ++i) put(sh.vv[(size_t)t * SITE_MAX_VV + i]);
    for (const SiteOff& o : sh.ob[t]) put(o);
    if (n_rows) *n_rows = k;
    return FKMC_OK;
}

int kmc_set_electrostatics(kmc_batch* b, const kmc_electrostatics* e)
{
    if (!b) return fail(FKMC_EINVAL, "null batch");
    if (!e) {
        if (!b->elec_on) return FKMC_OK;
        b->elec_on = false;
        b->elec_g.clear();
        b->elec_umax = 0;
        b->field_valid = false;
        {
            const int rc_ = drop_resident_cache(b);
            if (rc_) return rc_;
        }
        drop_window_graph(b);
        CK(run_pass_blocks(site_path(b) ? FKMC_PLAIN : b->opts.precision, b->cap, site_path(b), b->grains_on,
                           &b->run_blocks),
           "occupancy query");
        if (b->rates_set) {
            int rc = site_path(b) ? build_btab(b) : FKMC_OK;
            if (!rc) rc = plan_residency(b);
            if (!rc) rc = upload_desc(b);
            if (rc) return rc;
        }
        return FKMC_OK;
    }
    if (b->opts.precision != FKMC_PLAIN) return fail(FKMC_EINVAL, "electrostatics need the plain form");
    if (!(e->eps_r > 0.0) || !(e->eps_r <= 1e6) || !std::isfinite(e->q_vac) || std::fabs(e->q_vac) > 8.0 ||
        e->cycles < 1 || e->cycles > 200 || e->warm_cycles < 0 || e->warm_cycles > 200 || e->refresh_windows < 0)
        return fail(FKMC_EINVAL,
                    "electrostatics: eps_r in (0, 1e6], |q| <= 8, 1..200 cycles, 0..200 warm cycles, refresh >= 0");
    for (int r = 0; r < b->n; ++r)
        if (b->desc[r].nsite / 3 > INT32_MAX)
            return fail(FKMC_EINVAL, "electrostatics: at most 2^31 - 1 cells per replica");
    // buffers: u per site, tables, the multigrid levels of the largest replica
    int64_t total = 0, nodes = 0;
    for (int r = 0; r < b->n; ++r) {
        const MgPlan p = mg_plan(b->desc[r].L[0], b->desc[r].L[1], b->desc[r].L[2]);
        total = std::max(total, p.total);
        nodes = std::max<int64_t>(nodes, b->desc[r].nsite / 3);
    }
    if (!b->elec_u) b->elec_u = (int32_t*)b->dalloc(sizeof(int32_t) * b->nsite_total);
    if (!b->d_elec_g) b->d_elec_g = (int32_t*)b->dalloc(sizeof(int32_t) * 24 * b->n);
    if (!b->d_umax) b->d_umax = (unsigned*)b->dalloc(sizeof(unsigned));
    if (!b->field) b->field = (int32_t*)b->dalloc(sizeof(int32_t) * b->nsite_total);
    if (total > b->mg_total || nodes > b->mg_nodes) {
        for (void* q : {(void*)b->mgb.phi, (void*)b->mgb.f, (void*)b->mgb.r, (void*)b->mgb.e, (void*)b->mgb.g,
                        (void*)b->mgb.s, (void*)b->mgb.cnt})
            b->dfree(q);
        b->mgb.phi = (double*)b->dalloc(sizeof(double) * nodes);
        b->mgb.f = (double*)b->dalloc(sizeof(double) * nodes);
        b->mgb.r = (double*)b->dalloc(sizeof(double) * nodes);
        b->mgb.e = (float*)b->dalloc(sizeof(float) * total);
        b->mgb.g = (float*)b->dalloc(sizeof(float) * total);
        b->mgb.s = (float*)b->dalloc(sizeof(float) * total);
        b->mgb.cnt = (int32_t*)b->dalloc(sizeof(int32_t) * nodes);
        b->mg_total = total;
        b->mg_nodes = nodes;
    }
    if (!b->phi_prev) b->phi_prev = (double*)b->dalloc(sizeof(double) * b->ncell_total);
    if (!b->mgb.part) b->mgb.part = (double*)b->dalloc(sizeof(double) * MG_PARTIALS);
    if (!b->mgb.scalar) b->mgb.scalar = (double*)b->dalloc(sizeof(double) * 2);
    if (!b->elec_u || !b->d_elec_g || !b->d_umax || !b->field || !b->phi_prev || !b->mgb.phi || !b->mgb.f || !b->mgb.r ||
        !b->mgb.e || !b->mgb.g || !b->mgb.s || !b->mgb.cnt || !b->mgb.part || !b->mgb.scalar)
        return fail(FKMC_ENOMEM, "device allocation failed (electrostatics)");
    b->elec = *e;
    b->phi_prev_valid = false;  // the first solve starts from zero
    // own-potential tables: a unit charge on a site of each type, its 8 neighbours
    b->elec_g.assign(24 * (size_t)b->n, 0);
    for (int r = 0; r < b->n; ++r) {
        const RepDesc& D = b->desc[r];
        const MgPlan p = mg_plan(D.L[0], D.L[1], D.L[2]);
        const double scale = 1.602176634e-19 / (8.8541878128e-12 * e->eps_r * b->a_ang[r] * 1e-10);
        const int nx = D.L[0], ny = D.L[1], nz = D.L[2];
        std::vector<double> phi((size_t)nx * ny * nz);
        auto node = [&](int x, int y, int z) {
            x = ((x % nx) + nx) % nx;
            y = ((y % ny) + ny) % ny;
            z = ((z % nz) + nz) % nz;
            return phi[((size_t)z * ny + y) * nx + x];
        };
        auto site_phi = [&](int t, int x, int y, int z) {
            return 0.5 * (node(x, y, z) + node(x + (t == 0), y + (t == 1), z + (t == 2)));
        };
        for (int t = 0; t < 3; ++t) {
            CK(elec_solve_unit(D, t, scale, e->cycles, p, b->mgb, b->st), "unit-charge solve");
            CK(cudaMemcpyAsync(phi.data(), b->mgb.phi, sizeof(double) * phi.size(), cudaMemcpyDeviceToHost, b->st),
               "copy");
            CK(cudaStreamSynchronize(b->st), "synchronize");
            const int x = nx / 2, y = ny / 2, z = nz / 2;
            const double ps = site_phi(t, x, y, z);
            for (int n = 0; n < 8; ++n) {
                const NbEntry& nb = b->nbt.e[t][n];
                const double pj = site_phi(nb.t2, x + nb.dc[0], y + nb.dc[1], z + nb.dc[2]);
                b->elec_g[24 * (size_t)r + 8 * t + n] = (int32_t)std::llrint(e->q_vac * e->q_vac * (pj - ps) * 1e4);
            }
        }
    }
    CK(cudaMemcpyAsync(b->d_elec_g, b->elec_g.data(), sizeof(int32_t) * b->elec_g.size(), cudaMemcpyHostToDevice,
                       b->st),
       "table upload");
    b->elec_on = true;
    b->elec_umax = 0;
    b->field_valid = false;  // rebuilt with u at the next run
    {
        const int rc_ = drop_resident_cache(b);
        if (rc_) return rc_;
    }
    int rc = elec_refresh(b);
    if (rc) return rc;
    drop_window_graph(b);
    CK(run_pass_blocks(FKMC_PLAIN, b->cap, true, b->grains_on, &b->run_blocks), "occupancy query");
    if (b->rates_set) {
        rc = build_btab(b);
        if (!rc) rc = plan_residency(b);
        if (!rc) rc = upload_desc(b);
        if (rc) return rc;
    }
    CK(cudaStreamSynchronize(b->st), "synchronize");
    return FKMC_OK;
}

int kmc_solve_potential(kmc_batch* b, int32_t r, double* phi, size_t n, double* resid_rel)
{
    NvtxRange nvtx_range("kmc_solve_potential");
    if (!valid_replica(b, r) || !phi) return fail(FKMC_EINVAL, "bad replica or output");
    if (!b->elec_on) return fail(FKMC_ESTATE, "electrostatics are off");
    const RepDesc& D = b->desc[r];
    if ((int64_t)n != D.nsite / 3) return fail(FKMC_EINVAL, "n must equal nx ny nz");
    const MgPlan p = mg_plan(D.L[0], D.L[1], D.L[2]);
    const double scale = 1.602176634e-19 / (8.8541878128e-12 * b->elec.eps_r * b->a_ang[r] * 1e-10);
    double res = 0.0;
    CK(elec_solve(D, b->recs, b->counts, b->cap, b->n_vac[r], b->elec.q_vac, scale, b->elec.cycles, p, b->mgb, &res,
                  nullptr, nullptr, b->st),
       "potential solve");
    CK(cudaMemcpyAsync(phi, b->mgb.phi, sizeof(double) * n, cudaMemcpyDeviceToHost, b->st), "copy");
    CK(cudaStreamSynchronize(b->st), "synchronize");
    if (resid_rel) *resid_rel = res;
    return FKMC_OK;
}

int kmc_read_potential_energy(kmc_batch* b, int32_t r, int32_t* u, size_t n, int32_t* g)
{
    if (!valid_replica(b, r) || !u) return fail(FKMC_EINVAL, "bad replica or output");
    if (!b->elec_on) return fail(FKMC_ESTATE, "electrostatics are off");
    const RepDesc& D = b->desc[r];
    if ((int64_t)n != D.nsite) return fail(FKMC_EINVAL, "n must equal 3 nx ny nz");
    CK(cudaMemcpyAsync(u, b->elec_u + D.site_off, sizeof(int32_t) * n, cudaMemcpyDeviceToHost, b->st), "copy");
    CK(cudaStreamSynchronize(b->st), "synchronize");
    if (g) std::memcpy(g, b->elec_g.data() + 24 * (size_t)r, sizeof(int32_t) * 24);
    return FKMC_OK;
}

int kmc_write_potential_energy(kmc_batch* b, int32_t r, const int32_t* u, size_t n, const int32_t* g)
{
    if (!valid_replica(b, r) || !u) return fail(FKMC_EINVAL, "bad replica or input");
    if (!b->elec_on) return fail(FKMC_ESTATE, "electrostatics are off");
    const RepDesc& D = b->desc[r];
    if ((int64_t)n != D.nsite) return fail(FKMC_EINVAL, "n must equal 3 nx ny nz");
    int64_t um = 0;
    for (size_t i = 0; i < n; ++i) um = std::max<int64_t>(um, u[i] < 0 ? -(int64_t)u[i] : u[i]);
    CK(cudaMemcpyAsync(b->elec_u + D.site_off, u, sizeof(int32_t) * n, cudaMemcpyHostToDevice, b->st), "upload");
    if (g) {
        std::memcpy(b->elec_g.data() + 24 * (size_t)r, g, sizeof(int32_t) * 24);
        CK(cudaMemcpyAsync(b->d_elec_g + 24 * (size_t)r, g, sizeof(int32_t) * 24, cudaMemcpyHostToDevice, b->st),
           "upload");
    }
    CK(cudaStreamSynchronize(b->st), "synchronize");
    b->field_valid = false;
    {
        const int rc_ = drop_resident_cache(b);
        if (rc_) return rc_;
    }
    b->elec_age = 0;
    b->elec_umax = 0;  // re-derive the tables' range from what was written
    const int64_t keep = um;
    int rc = elec_cover(b, keep);
    if (rc) return rc;
    if (b->rates_set) {
        rc = build_btab(b);  // g may have grown the bound too
        if (!rc) rc = upload_desc(b);
        if (rc) return rc;
        drop_window_graph(b);
    }
    return FKMC_OK;
}

int kmc_set_grains(kmc_batch* b, const kmc_grains* g)
{
    if (!b) return fail(FKMC_EINVAL, "null batch");
    const bool on = g && g->n_grains > 1;
    if (on && b->opts.schedule == 2)
        return fail(FKMC_EINVAL, "grains need the colour-phase kernels (schedule 0 or 1)");
    if (on) {
        if (g->n_grains > 4096 || g->width < 1 || !(g->barrier_eV >= 0.0) || !(g->barrier_eV <= 10.0))
            return fail(FKMC_EINVAL, "grains: 2..4096 seeds, width >= 1, barrier in [0, 10] eV");
        for (int r = 0; r < b->n; ++r)
            for (int d = 0; d < 3; ++d)
                if (b->desc[r].L[d] < 2 * g->width + 1)
                    return fail(FKMC_EINVAL, "grains: every dimension must be >= 2 width + 1 cells");
        if (!b->grain) {
            b->grain = (int32_t*)b->dalloc(sizeof(int32_t) * b->ncell_total);
            b->gbound = (uint8_t*)b->dalloc((size_t)b->ncell_total);
            if (!b->grain || !b->gbound) return fail(FKMC_ENOMEM, "device allocation failed (grains)");
        }
        const int64_t need = 3 * (int64_t)b->n * g->n_grains;
        if (need > b->gX_len) {
            b->dfree(b->gX);
            b->gX = (int64_t*)b->dalloc(sizeof(int64_t) * need);
            b->gX_len = b->gX ? need : 0;
            if (!b->gX) return fail(FKMC_ENOMEM, "device allocation failed (grain seeds)");
        }
        CK(launch_grains(b->d_desc, b->n, b->ncell_total, g->n_grains, g->width, b->gX, b->grain, b->gbound, b->st),
           "grain kernels");
        b->grains = *g;
    }
    if (!on && !b->grains_on) return FKMC_OK;
    b->grains_on = on;
    drop_window_graph(b);
    CK(run_pass_blocks(site_path(b) ? FKMC_PLAIN : b->opts.precision, b->cap, site_path(b), on, &b->run_blocks),
       "occupancy query");
    if (b->rates_set) {
        for (int r = 0; r < b->n; ++r) {
            int rc = grain_tables(b, r);
            if (rc) return rc;
        }
        int rc = plan_residency(b);
        if (rc) return rc;
        rc = upload_desc(b);
        if (rc) return rc;
    }
    CK(cudaStreamSynchronize(b->st), "synchronize");
    return FKMC_OK;
}

int kmc_read_grains(kmc_batch* b, int32_t r, int32_t* grain, uint8_t* boundary, size_t n)
{
    if (!valid_replica(b, r) || !grain || !boundary) return fail(FKMC_EINVAL, "bad replica or output");
    if (!b->grains_on) return fail(FKMC_ESTATE, "grains are off");
    const RepDesc& D = b->desc[r];
    if ((int64_t)n != D.nsite / 3) return fail(FKMC_EINVAL, "n must equal nx ny nz");
    CK(cudaMemcpyAsync(grain, b->grain + D.site_off / 3, sizeof(int32_t) * n, cudaMemcpyDeviceToHost, b->st),
       "grain copy");
    CK(cudaMemcpyAsync(boundary, b->gbound + D.site_off / 3, n, cudaMemcpyDeviceToHost, b->st), "grain copy");
    CK(cudaStreamSynchronize(b->st), "synchronize");
    return FKMC_OK;
}

int kmc_read_dopants(kmc_batch* b, int32_t r, uint8_t* host_cells, size_t n)
{
    if (!valid_replica(b, r) || !host_cells) return fail(FKMC_EINVAL, "bad replica or output");
    const RepDesc& D = b->desc[r];
    if ((int64_t)n != D.nsite / 3) return fail(FKMC_EINVAL, "n must equal nx ny nz");
    if (!b->fe) {
        std::memset(host_cells, 0, n);
        return FKMC_OK;
    }
    CK(cudaMemcpyAsync(host_cells, b->fe + D.site_off / 3, n, cudaMemcpyDeviceToHost, b->st), "dopant copy");
    CK(cudaStreamSynchronize(b->st), "synchronize");
    return FKMC_OK;
}

int kmc_write_dopants(kmc_batch* b, int32_t r, const uint8_t* host_cells, size_t n)
{
    if (!valid_replica(b, r) || !host_cells) return fail(FKMC_EINVAL, "bad replica or input");
    const RepDesc& D = b->desc[r];
    if ((int64_t)n != D.nsite / 3) return fail(FKMC_EINVAL, "n must equal nx ny nz");
    if (!b->fe) {
        b->fe = (uint8_t*)b->dalloc((size_t)b->ncell_total);
        if (!b->fe) return fail(FKMC_ENOMEM, "device allocation failed");
        CK(cudaMemsetAsync(b->fe, 0, (size_t)b->ncell_total, b->st), "memset");
    }
    std::vector<uint8_t> h(n);
    int64_t cnt = 0;
    for (size_t c = 0; c < n; ++c) {
        h[c] = host_cells[c] ? 1 : 0;
        cnt += h[c];
    }
    CK(cudaMemcpyAsync(b->fe + D.site_off / 3, h.data(), n, cudaMemcpyHostToDevice, b->st), "dopant upload");
    CK(cudaStreamSynchronize(b->st), "synchronize");
    b->n_fe[r] = cnt;
    b->field_valid = false;
    {
        const int rc_ = drop_resident_cache(b);
        if (rc_) return rc_;
    }
    return FKMC_OK;
}

int kmc_read_site_field(kmc_batch* b, int32_t r, int32_t* host_field, size_t n)
{
    if (!valid_replica(b, r) || !host_field) return fail(FKMC_EINVAL, "bad replica or output");
    if (!site_path(b)) return fail(FKMC_ESTATE, "site energies are off");
    const RepDesc& D = b->desc[r];
    if ((int64_t)n != D.nsite) return fail(FKMC_EINVAL, "n must equal 3 nx ny nz");
    if (!b->field_valid) {
        int rc = rebuild_field(b);
        if (rc) return rc;
    }
    CK(cudaMemcpyAsync(host_field, b->field + D.site_off, sizeof(int32_t) * n, cudaMemcpyDeviceToHost, b->st),
       "field copy");
    CK(cudaStreamSynchronize(b->st), "synchronize");
    return FKMC_OK;
}

int kmc_check_invariants(kmc_batch* b, int32_t r, kmc_invariants* out)
{
    NvtxRange nvtx_range("kmc_check_invariants");
    if (!valid_replica(b, r) || !out) return fail(FKMC_EINVAL, "bad replica or output");
    if (!b->check_buf) {
        b->check_buf = (unsigned long long*)b->dalloc(sizeof(unsigned long long) * CHECK_WORDS);
        if (!b->check_buf) return fail(FKMC_ENOMEM, "device allocation failed");
    }
    CK(launch_check(b->desc[r], b->occ, b->recs, b->counts, b->cap, b->check_buf, b->st), "check kernels");
    unsigned long long h[CHECK_WORDS];
    CK(cudaMemcpyAsync(h, b->check_buf, sizeof h, cudaMemcpyDeviceToHost, b->st), "check copy");
    CK(cudaStreamSynchronize(b->st), "synchronize");
    std::memset(out, 0, sizeof *out);
    for (int c = 0; c < 4; ++c) out->sites[c] = (int64_t)h[CHK_SITES + c];
    out->records = (int64_t)h[CHK_RECORDS];
    out->rec_not_vacancy = (int64_t)h[CHK_NOT_VAC];
    out->rec_wrong_fragment = (int64_t)h[CHK_WRONG_FRAG];
    out->rec_outside = (int64_t)h[CHK_BAD_SITE];
    out->frag_bad_count = (int64_t)h[CHK_BAD_COUNT];
    out->hash_vac_sites = h[CHK_HASH_VAC];
    out->hash_rec_sites = h[CHK_HASH_REC];
    out->hash_rec_ids = h[CHK_HASH_ID];
    uint64_t ids = 0;  // every id 0 .. n_vac-1 once
    for (int64_t i = 0; i < b->n_vac[r]; ++i) ids += check_mix64((uint64_t)i);
    out->hash_ids_expected = ids;
    out->ok = out->sites[FKMC_V] == b->n_vac[r] && out->sites[FKMC_H] == b->n_H[r] && out->sites[3] == 0 &&
              out->records == b->n_vac[r] && out->rec_not_vacancy == 0 && out->rec_wrong_fragment == 0 &&
              out->rec_outside == 0 && out->frag_bad_count == 0 && out->hash_vac_sites == out->hash_rec_sites &&
              out->hash_rec_ids == ids;
    return FKMC_OK;
}

int kmc_get_replica_info(kmc_batch* b, int32_t r, kmc_replica_info* out)
{
    if (!valid_replica(b, r) || !out) return fail(FKMC_EINVAL, "bad replica or output");
    const RepDesc& D = b->desc[r];
    std::memset(out, 0, sizeof *out);
    for (int d = 0; d < 3; ++d) out->nfrag[d] = D.nf[d];
    out->cap_v = b->cap;
    out->F = D.F;
    out->precision = b->opts.precision;
    out->tau = D.tau;
    out->theta_tau = D.theta_tau;
    for (int i = 0; i < 6; ++i) {
        out->k64[i] = D.k64[i];
        out->q[i] = D.q[i];
    }
    out->window = D.window;
    out->hops = b->stats_host[2 * r];
    out->handoffs = b->stats_host[2 * r + 1];
    out->nsite = D.nsite;
    out->n_vac = b->n_vac[r];
    out->n_H = b->n_H[r];
    out->null_steps = D.null_step;
    out->null_theta = b->theta_host[r];
    out->null_time_s = null_time(b, r);
    out->n_Fe = b->n_fe[r];
    if ((int)b->run_kernel.size() == b->n) {
        out->kernel = b->run_kernel[r];
        out->ctas = b->run_ctas[r];
        out->draw_phases = b->run_kernel[r] == 1 ? D.pre_g : 0;
        out->draw_events = b->run_kernel[r] == 1 ? (D.pre_ev == 4 ? 4 : 2) : 0;
    }
    return FKMC_OK;
}

int32_t kmc_num_replicas(const kmc_batch* b) { return b ? b->n : 0; }

int kmc_destroy(kmc_batch* b)
{
    if (!b) return FKMC_OK;
    if (b->st) cudaStreamSynchronize(b->st);
    else cudaDeviceSynchronize();
    b->release();
    delete b;
    return FKMC_OK;
}

}  // extern "C"
