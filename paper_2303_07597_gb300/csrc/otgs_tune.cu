// otgs_tune.cu -- choice of the work decomposition by measurement.
//
// The plan's shape parameters decide how the (class group x target column)
// blocks of Sec. 2.3 are tiled over the evaluation kernel's CTAs: the panel
// height (rows of whole groups per work item, times 256 columns), the split
// height (groups taller than it are cut into pieces summed by several CTAs)
// and the stage fill (stages end early rather than cut a short group).
// Which shape is fastest depends on the distribution of group sizes and on
// the number of columns: short groups want tall panels (fewer, larger
// items), a few huge groups want pieces (no single item sets the kernel's
// duration).  The tuner times dense evaluations of the handle's own problems
// at a given point for each candidate shape, keeps the fastest, and
// remembers it for the process under a key made of the group-size histogram
// and the column and row counts, so handles of the same shape skip the
// measurement.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <map>
#include <mutex>
#include <string>
#include <vector>

#include "otgs_handle.cuh"

namespace otgs {

namespace {

std::mutex g_tune_mu;
std::map<std::string, PlanParams> g_tune_cache;

int log2_bucket(double v) { return v <= 1.0 ? 0 : (int)std::ceil(std::log2(v)); }

// Shape key: the share of rows in groups of each size class (2^k), in
// sixteenths, plus the size classes of the mean column count of a problem,
// of the total row count and of the number of problems.
std::string shape_key(const Handle* h)
{
    const HostPlan& hp = h->hp;
    std::vector<double> rows(24, 0.0);
    for (int32_t l = 0; l < hp.L; l++) {
        const int g = hp.goff[l + 1] - hp.goff[l];
        if (g > 0) rows[std::min(23, log2_bucket(g))] += g;
    }
    std::string key;
    for (int k = 0; k < 24; k++) {
        const int q = (int)std::lround(16.0 * rows[k] / (double)std::max<int64_t>(1, hp.m));
        key += std::to_string(q) + ",";
    }
    key += "|n" + std::to_string(log2_bucket((double)hp.n / hp.nprob));
    key += "|m" + std::to_string(log2_bucket((double)hp.m));
    key += "|p" + std::to_string(log2_bucket((double)hp.nprob));
    return key;
}

}  // namespace

}  // namespace otgs

using namespace otgs;

extern "C" {

int ot_gs_set_plan(ot_gs* hh, int32_t panel_rows, int32_t split_rows, int32_t stage_fill)
{
    if (!hh) return OTGS_EINVAL;
    Handle* h = reinterpret_cast<Handle*>(hh);
    if ((panel_rows != 0 && (panel_rows < 32 || panel_rows > 4096)) ||
        (split_rows != 0 && (split_rows < 64 || split_rows > 8192)) || stage_fill < 0 || stage_fill > 32) {
        h->fail(OTGS_EINVAL,
                "need panel_rows in [32, 4096], split_rows in [64, 8192] (or 0: default), stage_fill in [0, 32]");
        return OTGS_EINVAL;
    }
    PlanParams pp;
    pp.panel_rows = panel_rows;
    pp.split_rows = split_rows;
    pp.stage_fill = stage_fill;
    return h->setup_plan(pp) ? OTGS_OK : h->last_code;
}

int ot_gs_get_plan(const ot_gs* hh, int32_t* panel_rows, int32_t* split_rows, int32_t* stage_fill, int64_t* n_items)
{
    if (!hh) return OTGS_EINVAL;
    const Handle* h = reinterpret_cast<const Handle*>(hh);
    if (panel_rows) *panel_rows = h->hp.panel_height;
    if (split_rows) *split_rows = h->hp.split_height;
    if (stage_fill) *stage_fill = h->hp.stage_fill;
    if (n_items) *n_items = h->hp.nitems();
    return OTGS_OK;
}

int ot_gs_autotune(ot_gs* hh, const double* alpha, const double* beta, int32_t evals, int32_t* panel_rows,
                   int32_t* split_rows, int32_t* stage_fill, double* best_ms)
{
    if (!hh) return OTGS_EINVAL;
    Handle* h = reinterpret_cast<Handle*>(hh);
    if (!alpha || !beta || evals < 1) {
        h->fail(OTGS_EINVAL, "need alpha, beta and evals >= 1");
        return OTGS_EINVAL;
    }
    const std::string key = shape_key(h);
    PlanParams best;
    bool cached = false;
    {
        std::lock_guard<std::mutex> lk(g_tune_mu);
        auto it = g_tune_cache.find(key);
        if (it != g_tune_cache.end()) {
            best = it->second;
            cached = true;
        }
    }
    double best_t = 0.0;
    if (!cached) {
        double* D = (double*)h->dalloc(sizeof(double) * (size_t)h->nprob, "tuning objectives");
        if (!D) return h->last_code;
        cudaEvent_t e0, e1;
        if (!h->ck(cudaEventCreate(&e0), "cudaEventCreate")) return OTGS_ECUDA;
        if (!h->ck(cudaEventCreate(&e1), "cudaEventCreate")) {
            cudaEventDestroy(e0);
            return OTGS_ECUDA;
        }
        const int panels[] = {32, 64, 128, 256, 512, 1024};
        const int splits[] = {128, 256, 512, 1024};
        const int fills[] = {0, 16};
        best_t = INFINITY;
        bool ok = true;
        for (int pr : panels) {
            for (int q = 0; q < 8; q++) {
                const int sr = splits[q % 4], sf = fills[q / 4];
                if (sr < pr / 2) continue;  // pieces much shorter than a panel only add items
                PlanParams pp;
                pp.panel_rows = pr;
                pp.split_rows = sr;
                pp.stage_fill = sf;
                if (!h->setup_plan(pp)) { ok = false; break; }
                ok = h->eval_batch(alpha, beta, D, nullptr);  // warm-up
                ok = ok && h->ck(cudaEventRecord(e0, h->st), "cudaEventRecord");
                for (int e = 0; ok && e < evals; e++) ok = h->eval_batch(alpha, beta, D, nullptr);
                ok = ok && h->ck(cudaEventRecord(e1, h->st), "cudaEventRecord") &&
                     h->ck(cudaEventSynchronize(e1), "cudaEventSynchronize");
                float ms = 0.f;
                ok = ok && h->ck(cudaEventElapsedTime(&ms, e0, e1), "cudaEventElapsedTime");
                if (!ok) break;
                const double t = (double)ms / evals;
                if (t < best_t) {
                    best_t = t;
                    best = pp;
                }
            }
            if (!ok) break;
        }
        cudaEventDestroy(e0);
        cudaEventDestroy(e1);
        if (!ok) return h->last_code ? h->last_code : OTGS_ECUDA;
        std::lock_guard<std::mutex> lk(g_tune_mu);
        g_tune_cache[key] = best;
    }
    if (!h->setup_plan(best)) return h->last_code;
    if (panel_rows) *panel_rows = h->hp.panel_height;
    if (split_rows) *split_rows = h->hp.split_height;
    if (stage_fill) *stage_fill = h->hp.stage_fill;
    if (best_ms) *best_ms = cached ? 0.0 : best_t;
    return OTGS_OK;
}

int ot_gs_autotune_clear_cache(void)
{
    std::lock_guard<std::mutex> lk(g_tune_mu);
    g_tune_cache.clear();
    return OTGS_OK;
}

}  // extern "C"
