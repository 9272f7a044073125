// otgs_handle.cuh -- the state behind an ot_gs* handle.
#pragma once

#include <string>
#include <vector>

#include "otgs_internal.cuh"

namespace otgs {

struct Solver;
struct Batch;
void destroy_batch(Batch* b);
void set_create_error(const std::string& msg);  // the message ot_gs_last_error(NULL) returns

struct Handle {
    cudaStream_t st = nullptr;
    int64_t m = 0, n = 0;
    int32_t L = 0, ntiles = 0, unit_words = 0;
    ot_gs_params prm;
    HostPlan hp;
    DevPlan dp;
    std::vector<void*> allocs;
    std::string err;
    int last_code = 0;
    bool st_synced_ok = false;

    // problems: one, or a batch of independent ones concatenated (rows in
    // problem order, class-sorted within a problem; columns in problem order)
    int32_t nprob = 1;
    bool shard = false;               // a column shard: b is a slice of the marginal (no solve)
    std::vector<ProbDesc> probs_h;    // per problem: C (sorted rows), ldc, sizes, offsets
    ProbDesc* probs = nullptr;        // device copy
    std::vector<BProb> bprob_h;       // per problem: offsets and work-item range (plan-dependent)
    BProb* bprob = nullptr;           // device copy
    Batch* batch = nullptr;           // batched solver state (first ot_gs_batch_solve)
    FxScale* pfx = nullptr;           // per problem: fixed-point scale of the last batch evaluation point
    CUtensorMap* maps = nullptr;      // device: per problem, TMA descriptors (box[], then tile[])
    TmaMaps tm0;                      // problem 0's descriptors (passed in the kernel's parameters when nprob == 1)
    PlanParams plan_params;           // the parameters of the current plan (0 = defaults)
    int plan_gen = 0;                 // bumped by every (re)build of the plan
    std::vector<int32_t> labels_h;    // all problems' labels (caller order), for re-planning
    std::vector<int64_t> pm_h, pn_h;
    std::vector<int32_t> pL_h;
    std::vector<void*> plan_allocs;   // device buffers sized by the plan (replaced on re-planning)
    double* a_sorted = nullptr;
    double* b = nullptr;
    float cmax = 0.f;

    // one evaluation
    float4* rowA = nullptr;         // sorted rows: (alpha hi, lo, bound_up(hi), 0)
    float2* B2 = nullptr;           // (beta hi, lo), per problem from probs_h[k].bcoff
    EvalCtl* ctl = nullptr;         // evaluation control word (work counter, scale maxima)
    int* kerr = nullptr;            // evaluation kernel error word
    int n_sm = 0;
    double* alpha_eval = nullptr;   // sorted alpha of the last evaluation
    unsigned long long* rowfx = nullptr;  // fixed-point row sums of T
    unsigned long long* colfx = nullptr;  // fixed-point column sums of T
    unsigned long long* psix = nullptr;  // per problem of a batch: psi of the exact-sum kernel (hi, lo)
    XEntry* xent = nullptr;         // flagged block sets for the exact-sum kernel (sized by the plan):
    XEntry* xtall = nullptr;        // classes of at most XTALL_ROWS rows, taller classes
    int32_t xent_cap = 0, xtall_cap = 0;
    uint32_t* xtmap = nullptr;      // transposed route: column task of a taller class -> its set
    int32_t xtcol_cap = 0;
    unsigned long long* fcount = nullptr;  // flagged blocks (statistics)
    int64_t dbg_stall_ns = 0;       // test hooks (ot_gs_debug): a stalled ring with this wait limit,
    int64_t dbg_nan_eval = 0;       //   a solve's objective NaN from this evaluation on,
    int64_t dbg_route = 0;          //   a screened evaluation's route (0: chosen, 1: bound pass, 2: block sets)
    float* split_part = nullptr;    // partial block sums of the pieces of split groups
    int nred = 0;
    double* block_part = nullptr;
    unsigned* counter = nullptr;
    double* scal = nullptr;
    double* host_scal = nullptr;

    // screening (Sec. 3): allocated on first use
    bool screen_alloc = false;
    bool snap_valid = false;      // zt/ot/alpha_snap/beta_snap describe a snapshot
    float* zt = nullptr;          // z~ (rounded up), L x ntiles*TW
    float* zt_tile = nullptr;     // L x ntiles: the largest z~ of each 32-column tile (+inf with a NaN)
    float* ot = nullptr;          // o~, L x ntiles*TW
    double* alpha_snap = nullptr; // sorted
    double* beta_snap = nullptr;
    uint32_t* Nmask = nullptr;    // set N, one word per unit (bit = column within tile)
    uint32_t* skipmask = nullptr; // last screened evaluation's skip decisions, same layout
    uint32_t* unit_need = nullptr;// L x unit_words
    uint8_t* item_active = nullptr;
    uint8_t* stage_m8 = nullptr;  // [nstages][STAGE_ROWS]: per row, the needed tiles of its item
    uint32_t* stage_need = nullptr; // [ceil(nstages / 32)]: stages with a needed row
    float* gstat = nullptr;       // per group: npos, nabs, nneg, theta_skip
    float2* drow = nullptr;       // per sorted row: RU([alpha - alpha~]_+), RN(alpha - alpha~) as FP32
    float* cstat = nullptr;       // per column: dbp, dbabs, dbneg (an array each); per tile: max dbp
    unsigned* gmax = nullptr;     // float bits: max|alpha|, max|beta|, max|alpha~|, max|beta~|
    unsigned long long* dcount = nullptr; // device counters: in_N, checked, skipped, units
    float* sg_ru = nullptr;       // sqrt(g_l) rounded up
    float* sg_rn = nullptr;       // sqrt(g_l) rounded to nearest
    int64_t dense_units = 0;      // units streamed by dense passes
    double dense_cbytes = 0.0;    // bytes of C streamed by dense passes
    ot_gs_stats stats_host;

    // optional event timing of evaluation-kernel launches
    bool timing = false;
    std::vector<cudaEvent_t> ev_pool;
    size_t ev_used = 0;
    int eval_launch(const EvalArgs& e, int n_ctas);  // returns the kernels launched

    ~Handle();
    bool init(int32_t nprob, const float* const* C, const int64_t* ldc, const double* const* a,
              const double* const* b, const int32_t* const* labels, const int64_t* m, const int64_t* n,
              const int32_t* L, double gamma, double mu, cudaStream_t st);
    // (re)builds the work decomposition with the given parameters and the buffers sized by it
    bool setup_plan(const PlanParams& pp);
    void* plan_alloc(size_t bytes, const char* what);
    void free_plan();
    bool fail(int code, const std::string& msg);
    bool ck(cudaError_t e, const char* what);
    void* dalloc(size_t bytes, const char* what);

    EvalArgs eval_args(const uint8_t* active, const uint32_t* need, bool snap);
    void prep(const double* alpha, bool alpha_sorted, const double* beta);
    ReduceArgs reduce_args(const uint8_t* active, double* out_caller, double* G_sorted, const double* dir,
                           const double* beta_ptr);
    bool eval_dense(const double* alpha, bool alpha_sorted, const double* beta, double* out_caller,
                    double* G_sorted, const double* dir, bool snap);
    // evaluations whose preparation (rowA, B2, alpha_eval, ctl) is already in place
    bool eval_dense_prepped(const double* beta, double* G_sorted, const double* dir);
    bool eval_dense_core(const double* beta, double* out_caller, double* G_sorted, const double* dir, bool snap);
    bool eval_screened_prepped(const double* beta, double* G_sorted, const double* dir,
                               double* out_caller = nullptr);
    // every problem at (alpha, beta) in the caller's concatenated layout:
    // D [nprob] and the gradient [m + n] (may be NULL), device
    bool eval_batch(const double* alpha, const double* beta, double* D, double* grad);
    Solver* solver = nullptr;
    // While set (batched solver trials): evaluations are gated on this device
    // flag and are counted in the statistics by the solver afterwards.
    const int* eval_gate = nullptr;
    int64_t nonempty_units() const;
    void count_dense_evals(int64_t k);     // statistics of k dense evaluations
    void count_screened_evals(int64_t k);  // (block counts of screened ones come from the device)

    // screening (otgs_screen_host.cu)
    bool ensure_screen();
    bool zero_snapshot();
    void invalidate_screen() { snap_valid = false; }
    bool zt_tiles();  // zt_tile from zt (after every write of zt)
    bool snapshot_at(const double* alpha, bool alpha_sorted, const double* beta, bool build_N,
                     double* out_caller, double* G_sorted, const double* dir);
    bool eval_screened(const double* alpha, bool alpha_sorted, const double* beta, double* out_caller,
                       double* G_sorted, const double* dir);
    bool collect_stats();
    void reset_device_stats();
};

// The calls that take one problem's vectors reject batch handles.
inline bool single_problem(Handle* h)
{
    if (h->nprob == 1) return true;
    return h->fail(OTGS_EINVAL, "a batch of problems: use the ot_gs_batch_* calls");
}

}  // namespace otgs
