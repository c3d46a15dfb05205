// fkmc_kernels.h -- host-side launchers of the kernels in fkmc_kernels.cu.
#pragma once
#include <cuda_runtime.h>

#include "fkmc_device.cuh"

namespace fkmc {

// sets the thread-local message of kmc_last_error() and returns `code`
int set_error(int code, const char* msg);

cudaError_t upload_neighbours(const NbEntry* host24);
cudaError_t launch_init(const RepDesc& D, int b_bits, int64_t n_vac, int64_t n_total, uint32_t* occ,
                        VacRec* recs, int32_t* counts, int cap, uint32_t* status, cudaStream_t st);
size_t phase_smem_bytes(int cap, bool site);
cudaError_t phase_prepare(int cap);
cudaError_t run_pass_blocks(int prec, int cap, bool site, bool grain, int* blocks);
cudaError_t small_pass_blocks(int prec, bool grain, int lane, int* blocks);
constexpr int64_t SPLIT_MIN_ITEMS = 32768;  // fragments per phase from which the small-fragment pass runs
constexpr int ACT_COUNTERS = 32;  // act_count: 3 active lists x 8 phases, 8 window tickets
constexpr int LANE_MAX_V = 8;      // vacancies per fragment of the persistent one-thread-per-fragment pass
constexpr int LANE_REG_MAX_V = 4;  // ... of its register form
constexpr int64_t LANE_PERSIST_ITEMS = 1 << 19;  // fragments per phase from which the persistent form runs
constexpr int LANE_NONE = 0, LANE_REGISTERS = 1, LANE_PERSISTENT = 2;
// mode: kmc_opts.small_pass (0 auto, 1 always, 2 always and grouped, -1 never)
bool window_split(bool site, int64_t total_items, int mode);
// form of the one-thread-per-fragment pass (mixed form only; LANE_NONE: the
// grouped pass); form: kmc_opts.lane_form (0 auto, 1 registers, 2 persistent)
int window_lane(int prec, int mode, int form, int64_t total_items);
// act: 3 lists of total_items entries (general, one vacancy, two vacancies);
// act_count: ACT_COUNTERS counters (list l, phase p at 8 l + p; the window
// ticket of phase p of the one-thread-per-fragment pass at 24 + p)
// cls: total_items bytes (the screen's class of each item for the register form)
cudaError_t launch_window(int prec, const RepDesc* d_descs, int nrep, int64_t total_items,
                          unsigned long long* wctl, uint32_t* perms, ActEntry* act, int32_t* act_count,
                          uint8_t* cls, uint32_t* occ, VacRec* recs, int32_t* counts, int32_t* tracer,
                          unsigned long long* stats, uint32_t* status, int cap, int run_blocks,
                          int small_blocks, bool split, int lane_form, const SiteArgs& sa, cudaStream_t st,
                          cudaStream_t side, cudaEvent_t fork, cudaEvent_t join);
cudaError_t launch_grains(const RepDesc* d_descs, int nrep, int64_t ncell_total, int n_grains, int width, int64_t* X,
                          int32_t* grain, uint8_t* gb, cudaStream_t st);
cudaError_t launch_init_dopants(const RepDesc& D, int b_bits, int64_t n_fe, uint8_t* fe, cudaStream_t st);
cudaError_t launch_site_field(const RepDesc* d_descs, int nrep, const VacRec* recs, const int32_t* counts,
                              int64_t nfrag_total, int cap, int64_t nsite_total, const uint8_t* fe,
                              const SiteOff* bo, int n_bo, const SiteArgs& sa, cudaStream_t st);
// atom-based fragment kMC with null events (fkmc_null.cu)
cudaError_t launch_null_gather(const RepDesc* d_descs, int nrep, const VacRec* recs, const int32_t* counts,
                               int64_t nfrag_total, int cap, VacRec* vac, uint32_t* status, cudaStream_t st);
cudaError_t launch_null_scatter(const RepDesc* d_descs, int nrep, int64_t total_vac, const VacRec* vac,
                                VacRec* recs, int32_t* counts, int64_t nfrag_total, int cap, uint32_t* status,
                                cudaStream_t st);
cudaError_t null_upload_neighbours(const NbEntry* host24);
cudaError_t launch_null_step(const RepDesc* d_descs, int nrep, int64_t total_vac, int64_t total_picks, VacRec* vac,
                             uint32_t* occ, const uint8_t* gb, unsigned long long* acc,
                             NullProp* props,
                             unsigned long long* claims, int32_t* tracer, double* theta, double* nE,
                             unsigned long long* stats, unsigned long long* nctl, cudaStream_t st);
cudaError_t launch_moments(const RepDesc& D, int species, const uint32_t* occ, const VacRec* recs,
                           const int32_t* counts, const int32_t* tracer, int cap,
                           unsigned long long* out, cudaStream_t st);

cudaError_t launch_moments_all(const RepDesc* d_descs, int nrep, const VacRec* recs, const int32_t* counts,
                               int64_t max_frag_per_replica, int cap, unsigned long long* out, cudaStream_t st);

// electrostatics of the mu-scale model (fkmc_poisson.cu): multigrid on the B-site grid
constexpr int MG_MAX_LEVELS = 16;
constexpr int MG_PARTIALS = 256;  // blocks of the deterministic reductions
struct MgPlan {
    int levels;
    int dim[MG_MAX_LEVELS][3];
    int64_t off[MG_MAX_LEVELS];  // first node of each level in the level-stacked buffers
    int64_t total;
};
struct MgBuffers {
    double* phi;     // [level-0 nodes] the potential (FP64)
    double* f;       // [level-0 nodes] right-hand side (FP64)
    double* r;       // [level-0 nodes] residual of the final check
    float* e;        // [total] FP32 correction per level
    float* g;        // [total] FP32 right-hand side per level (level 0: the FP64 defect, rounded)
    float* s;        // [total] FP32 residual (and the Jacobi scratch of an odd level)
    int32_t* cnt;    // [level-0 nodes] half-charge counts
    double* part;    // [MG_PARTIALS]
    double* scalar;  // [2]
};
MgPlan mg_plan(int nx, int ny, int nz);
int64_t mg_cycle_kernels(const MgPlan& p);  // kernel launches of one V-cycle
cudaError_t elec_solve(const RepDesc& D, const VacRec* recs, const int32_t* counts, int cap, int64_t n_vac,
                       double q, double scale, int cycles, const MgPlan& p, const MgBuffers& b, double* resid_rel,
                       const double* init, double* save, cudaStream_t st);
cudaError_t elec_solve_unit(const RepDesc& D, int t, double scale, int cycles, const MgPlan& p, const MgBuffers& b,
                            cudaStream_t st);
cudaError_t elec_update(const RepDesc& D, const double* phi, double q, int32_t* u, int32_t* field, unsigned* umax,
                        cudaStream_t st);
cudaError_t elec_add(int32_t* field, const int32_t* u, int64_t n, cudaStream_t st);

// Per-fragment event totals and dirty flags the resident kernels leave at the end
// of a call (batch-wide fragment index), and per replica whether they are still
// valid: the host clears `valid` whenever anything but a resident run changes a
// replica's state or rates, and the next call then starts from every fragment dirty.
struct ResCache {
    unsigned long long* tot;
    uint8_t* dirty;
    uint8_t* valid;
};

// cluster-resident kernel (fkmc_resident.cu): one replica per thread-block cluster,
// CTA c holding the z-slab of fragment layers [fz0[c], fz0[c+1])
constexpr int CLUSTER_MAX_CTAS = 16;
constexpr int CLUSTER_THREADS = 512;
struct ClusterPlan {
    int32_t rep;                          // replica index in the batch
    int32_t ncta;                         // CTAs of the cluster
    int32_t fz0[CLUSTER_MAX_CTAS + 1];    // fragment layers of CTA c: [fz0[c], fz0[c + 1])
    int32_t zs;                           // cells in z of the thickest slab (the common layout)
    int32_t nfl;                          // fragments of the thickest slab
    int32_t vcap;                         // vacancy slots per CTA
    int32_t icap;                         // inbox entries per phase parity per CTA
};
size_t cluster_smem_bytes(const RepDesc& D, const ClusterPlan& p, int cap);
// the plan with the fewest CTAs in [min_ctas, max_ctas] whose slabs fit one SM's shared memory
bool make_cluster_plan(const RepDesc& D, int64_t n_vac, int cap, int min_ctas, int max_ctas, ClusterPlan* out);
cudaError_t cluster_prepare();
int cluster_fits(int ncta, size_t smem);  // clusters of ncta CTAs with this much shared memory the GPU can hold at once
cudaError_t launch_cluster(const RepDesc* d_descs, const ClusterPlan* d_plans, int nplans, int ncta, size_t smem,
                           uint64_t windows, uint32_t* occ, VacRec* recs, int32_t* counts, int32_t* tracer,
                           unsigned long long* stats, uint32_t* status, int cap, const NbTable& nbt,
                           const ResCache& rc, cudaStream_t st);

// replica-resident kernel (fkmc_resident.cu)
constexpr int RESIDENT_MAX_SLOTS = 64;               // vacancies per fragment a thread can hold
constexpr size_t RESIDENT_MAX_SMEM = 220 * 1024;     // dynamic shared memory per replica CTA
size_t resident_smem_bytes(const RepDesc& D, int64_t n_vac, int cap, int threads, int pre_g, int pre_ev);
cudaError_t resident_prepare();
cudaError_t launch_resident(const RepDesc* d_descs, const int32_t* d_reps, int nreps, const int64_t* d_nvac,
                            size_t smem, int threads, int cluster, uint64_t windows, uint32_t* occ, VacRec* recs,
                            int32_t* counts, int32_t* tracer, unsigned long long* stats, uint32_t* status,
                            int cap, const NbTable& nbt, uint32_t stuck_wait_us, const ResCache& rc,
                            cudaStream_t st);

}  // namespace fkmc
