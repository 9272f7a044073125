// otgs_api.cu -- the C ABI (include/otgs.h): handle life cycle, validation,
// device buffers, and the host side of one evaluation.
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <string>
#include <vector>

#include "otgs_solver.cuh"

using namespace otgs;

static thread_local std::string g_create_error;

namespace otgs {

void set_create_error(const std::string& msg) { g_create_error = msg; }

bool Handle::fail(int code, const std::string& msg)
{
    err = msg;
    last_code = code;
    return false;
}

bool Handle::ck(cudaError_t e, const char* what)
{
    if (e == cudaSuccess) return true;
    err = std::string(what) + ": " + cudaGetErrorString(e);
    last_code = OTGS_ECUDA;
    return false;
}

void* Handle::dalloc(size_t bytes, const char* what)
{
    void* p = nullptr;
    if (bytes == 0) bytes = 16;
    cudaError_t e = cudaMalloc(&p, bytes);
    if (e != cudaSuccess) {
        err = std::string("cudaMalloc(") + what + ", " + std::to_string(bytes) + " B): " + cudaGetErrorString(e);
        last_code = e == cudaErrorMemoryAllocation ? OTGS_ENOMEM : OTGS_ECUDA;
        cudaGetLastError();
        return nullptr;
    }
    allocs.push_back(p);
    return p;
}

Handle::~Handle()
{
    if (st_synced_ok) cudaStreamSynchronize(st);
    delete solver;
    destroy_batch(batch);
    for (cudaEvent_t e : ev_pool) cudaEventDestroy(e);
    for (void* p : allocs) cudaFree(p);
    free_plan();
    if (host_scal) cudaFreeHost(host_scal);
}

template <class T>
static T* upload(Handle* h, const std::vector<T>& v, const char* what)
{
    T* d = (T*)h->dalloc(sizeof(T) * (v.empty() ? 1 : v.size()), what);
    if (!d) return nullptr;
    if (!v.empty() && !h->ck(cudaMemcpyAsync(d, v.data(), sizeof(T) * v.size(), cudaMemcpyHostToDevice, h->st), what))
        return nullptr;
    return d;
}

void* Handle::plan_alloc(size_t bytes, const char* what)
{
    void* p = dalloc(bytes, what);
    if (p) {
        allocs.pop_back();
        plan_allocs.push_back(p);
    }
    return p;
}

void Handle::free_plan()
{
    for (void* p : plan_allocs) cudaFree(p);
    plan_allocs.clear();
}

template <class T>
static T* plan_upload(Handle* h, const std::vector<T>& v, const char* what)
{
    T* d = (T*)h->plan_alloc(sizeof(T) * (v.empty() ? 1 : v.size()), what);
    if (!d) return nullptr;
    if (!v.empty() && !h->ck(cudaMemcpyAsync(d, v.data(), sizeof(T) * v.size(), cudaMemcpyHostToDevice, h->st), what))
        return nullptr;
    return d;
}

bool Handle::init(int32_t np, const float* const* C_, const int64_t* ldc_, const double* const* a_,
                  const double* const* b_, const int32_t* const* labels_, const int64_t* m_, const int64_t* n_,
                  const int32_t* L_, double gamma_, double mu_, cudaStream_t st_)
{
    st = st_;
    nprob = np;
    prm.gamma = gamma_; prm.mu = mu_;
    prm.r = 10; prm.lbfgs_m = 10; prm.use_screening = 0; prm.use_lower_bound = 1;
    prm.time_budget_ms = 0.0;
    prm.ftol = 0.0;
    // labels to the host, one array for all problems
    int64_t mtot = 0;
    for (int32_t k = 0; k < np; k++) mtot += m_[k];
    labels_h.resize(mtot);
    pm_h.assign(m_, m_ + np);
    pn_h.assign(n_, n_ + np);
    pL_h.assign(L_, L_ + np);
    {
        int64_t off = 0;
        for (int32_t k = 0; k < np; k++) {
            if (!ck(cudaMemcpyAsync(labels_h.data() + off, labels_[k], sizeof(int32_t) * m_[k],
                                    cudaMemcpyDeviceToHost, st),
                    "labels D2H"))
                return false;
            off += m_[k];
        }
    }
    if (!ck(cudaStreamSynchronize(st), "labels sync")) return false;
    st_synced_ok = true;
    {
        std::vector<const int32_t*> lp(np);
        int64_t off = 0;
        for (int32_t k = 0; k < np; k++) {
            lp[k] = labels_h.data() + off;
            off += m_[k];
        }
        std::string pe = build_plan_batch(np, lp.data(), m_, n_, L_, PlanParams(), hp);
        if (!pe.empty()) return fail(OTGS_EINVAL, pe);
    }
    m = hp.m; n = hp.n; L = hp.L;
    ntiles = hp.ntiles;
    unit_words = (ntiles + 31) / 32;
    auto where = [&](int32_t k) { return np == 1 ? std::string() : " (problem " + std::to_string(k) + ")"; };
    // validation of C, a, b on the device
    {
        double* sums = (double*)dalloc(2 * sizeof(double) * np, "check sums");
        int* flags = (int*)dalloc(4 * sizeof(int) * np, "check flags");
        if (!sums || !flags) return false;
        if (!ck(cudaMemsetAsync(sums, 0, 2 * sizeof(double) * np, st), "memset")) return false;
        if (!ck(cudaMemsetAsync(flags, 0, 4 * sizeof(int) * np, st), "memset")) return false;
        for (int32_t k = 0; k < np; k++)
            launch_check_finite(C_[k], ldc_[k], (int32_t)m_[k], (int32_t)n_[k], a_[k], b_[k], sums + 2 * k,
                                flags + 4 * k, st);
        std::vector<double> hs(2 * (size_t)np);
        std::vector<int> hf(4 * (size_t)np);
        if (!ck(cudaMemcpyAsync(hs.data(), sums, sizeof(double) * hs.size(), cudaMemcpyDeviceToHost, st), "check D2H"))
            return false;
        if (!ck(cudaMemcpyAsync(hf.data(), flags, sizeof(int) * hf.size(), cudaMemcpyDeviceToHost, st), "check D2H"))
            return false;
        if (!ck(cudaStreamSynchronize(st), "check sync")) return false;
        for (int32_t k = 0; k < np; k++) {
            const int* f = hf.data() + 4 * k;
            const double* sm = hs.data() + 2 * k;
            if (f[0]) return fail(OTGS_ENONFINITE, "C has a non-finite entry" + where(k));
            if (f[1]) return fail(OTGS_EINVAL, "C has a negative entry" + where(k));
            if (f[2]) return fail(OTGS_EINVAL, "a and b must be positive and finite" + where(k));
            if (!shard && !(std::fabs(sm[0] - sm[1]) <= 1e-12 * std::fmax(1.0, std::fmax(sm[0], sm[1]))))
                return fail(OTGS_EINVAL, "sum(a) != sum(b)" + where(k));
            unsigned cbits = (unsigned)f[3];
            float cm;
            memcpy(&cm, &cbits, sizeof(float));
            cmax = std::max(cmax, cm);
        }
    }
    dp.perm = upload(this, hp.perm, "perm");
    if (!dp.perm) return false;
    // C of each problem: borrowed when class-sorted and laid out as TMA needs
    // (16-byte aligned base and row stride), else a sorted, padded copy
    probs_h.resize(np);
    {
        std::vector<char> copy(np, 0);
        size_t copy_floats = 0;
        int64_t off = 0;
        for (int32_t k = 0; k < np; k++) {
            bool sorted = true;
            for (int64_t i = 1; i < m_[k] && sorted; i++) sorted = labels_h[off + i] >= labels_h[off + i - 1];
            const bool aligned = (reinterpret_cast<uintptr_t>(C_[k]) % 16 == 0) && (ldc_[k] % 4 == 0);
            copy[k] = !(sorted && aligned);
            if (copy[k]) copy_floats += (size_t)m_[k] * (size_t)((n_[k] + 3) / 4 * 4);
            off += m_[k];
        }
        float* Cs = nullptr;
        if (copy_floats) {
            Cs = (float*)dalloc(sizeof(float) * copy_floats, "sorted C");
            if (!Cs) return false;
        }
        size_t at = 0;
        for (int32_t k = 0; k < np; k++) {
            ProbDesc& pd = probs_h[k];
            memset(&pd, 0, sizeof(pd));
            pd.m = (int32_t)m_[k];
            pd.n = (int32_t)n_[k];
            pd.roff = hp.proff[k];
            pd.coff = hp.pcoff[k];
            pd.bcoff = hp.pbcoff[k];
            if (copy[k]) {
                const int64_t ld = (n_[k] + 3) / 4 * 4;
                launch_gather_rows(C_[k], ldc_[k], dp.perm + pd.roff, pd.roff, pd.m, pd.n, Cs + at, ld, st);
                pd.C = Cs + at;
                pd.ldc = ld;
                at += (size_t)m_[k] * (size_t)ld;
            } else {
                pd.C = C_[k];
                pd.ldc = ldc_[k];
            }
        }
    }
    {
        // the transposed copy: each block (l, j) is one contiguous run of rows
        size_t ct_floats = 0;
        for (int32_t k = 0; k < np; k++) ct_floats += (size_t)n_[k] * (size_t)((m_[k] + 3) / 4 * 4);
        float* CT = (float*)dalloc(sizeof(float) * std::max<size_t>(ct_floats, 1), "transposed C");
        if (!CT) return false;
        size_t at = 0;
        for (int32_t k = 0; k < np; k++) {
            ProbDesc& pd = probs_h[k];
            pd.ldct = (m_[k] + 3) / 4 * 4;
            pd.CT = CT + at;
            launch_transpose(pd.C, pd.ldc, pd.m, pd.n, CT + at, pd.ldct, st);
            at += (size_t)n_[k] * (size_t)pd.ldct;
        }
        if (!ck(cudaGetLastError(), "transpose")) return false;
    }
    probs = upload(this, probs_h, "problem table");
    if (!probs) return false;
    {
        std::vector<TmaMaps> tm(np);
        for (int32_t k = 0; k < np; k++) {
            std::string te = make_tmaps(probs_h[k].C, probs_h[k].ldc, probs_h[k].m, probs_h[k].n, tm[k]);
            if (!te.empty()) return fail(OTGS_ECUDA, te + where(k));
        }
        static_assert(sizeof(TmaMaps) == 2 * TMA_BOXES * sizeof(CUtensorMap), "maps are packed");
        maps = (CUtensorMap*)upload(this, tm, "TMA descriptors");  // cudaMalloc: 256-byte aligned
        if (!maps) return false;
        tm0 = tm[0];
    }
    // row groups (independent of the plan's parameters)
    dp.goff = upload(this, hp.goff, "goff");
    dp.rgroup = upload(this, hp.rgroup, "rgroup");
    dp.rowg = upload(this, hp.rowg, "row groups");
    if (!dp.goff || !dp.rgroup || !dp.rowg) return false;
    // marginals: a in sorted order, b concatenated
    a_sorted = (double*)dalloc(sizeof(double) * m, "a_sorted");
    b = (double*)dalloc(sizeof(double) * n, "b");
    if (!a_sorted || !b) return false;
    if (np == 1) {
        launch_permute_f64(a_[0], dp.perm, (int32_t)m, a_sorted, true, st);
    } else {
        double* acat = (double*)dalloc(sizeof(double) * m, "a (concatenated)");
        if (!acat) return false;
        for (int32_t k = 0; k < np; k++)
            if (!ck(cudaMemcpyAsync(acat + hp.proff[k], a_[k], sizeof(double) * m_[k], cudaMemcpyDeviceToDevice, st),
                    "a copy"))
                return false;
        launch_permute_f64(acat, dp.perm, (int32_t)m, a_sorted, true, st);
    }
    for (int32_t k = 0; k < np; k++)
        if (!ck(cudaMemcpyAsync(b + hp.pcoff[k], b_[k], sizeof(double) * n_[k], cudaMemcpyDeviceToDevice, st),
                "b copy"))
            return false;
    // evaluation buffers
    rowA = (float4*)dalloc(sizeof(float4) * (size_t)m, "rowA");
    B2 = (float2*)dalloc(sizeof(float2) * (size_t)hp.nb2, "B2");
    ctl = (EvalCtl*)dalloc(sizeof(EvalCtl), "evaluation control");
    kerr = (int*)dalloc(sizeof(int) * 4, "kernel error");
    alpha_eval = (double*)dalloc(sizeof(double) * m, "alpha_eval");
    rowfx = (unsigned long long*)dalloc(sizeof(unsigned long long) * (size_t)m, "row sums");
    colfx = (unsigned long long*)dalloc(sizeof(unsigned long long) * (size_t)n, "column sums");
    pfx = (FxScale*)dalloc(sizeof(FxScale) * (size_t)np, "per-problem fixed-point scales");
    if (!rowA || !B2 || !ctl || !kerr || !alpha_eval || !rowfx || !colfx || !pfx) return false;
    if (!ck(cudaMemsetAsync(B2, 0, sizeof(float2) * (size_t)hp.nb2, st), "memset B2")) return false;
    if (!ck(cudaMemsetAsync(kerr, 0, sizeof(int) * 4, st), "memset err")) return false;
    psix = (unsigned long long*)dalloc(sizeof(unsigned long long) * 2 * (size_t)np, "psi of the exact-sum kernel");
    if (!psix) return false;
    if (!ck(cudaMemsetAsync(psix, 0, sizeof(unsigned long long) * 2 * (size_t)np, st), "memset psix")) return false;
    {
        int dev = 0;
        if (!ck(cudaGetDevice(&dev), "cudaGetDevice")) return false;
        if (!ck(cudaDeviceGetAttribute(&n_sm, cudaDevAttrMultiProcessorCount, dev), "SM count")) return false;
    }
    fcount = (unsigned long long*)dalloc(sizeof(unsigned long long) * 2, "flagged block counters");
    if (!fcount) return false;
    if (!ck(cudaMemsetAsync(fcount, 0, sizeof(unsigned long long) * 2, st), "memset counters")) return false;
    if (!stream_prepare()) return fail(OTGS_ECUDA, "cudaFuncSetAttribute(evaluation kernel)");
    if (!setup_plan(PlanParams())) return false;
    nred = reduce_blocks((int32_t)m, (int32_t)n);
    block_part = (double*)dalloc(sizeof(double) * REDUCE_PARTS * (size_t)nred, "block_part");
    counter = (unsigned*)dalloc(sizeof(unsigned) * 4, "counter");
    scal = (double*)dalloc(sizeof(double) * 8, "scal");
    if (!block_part || !counter || !scal) return false;
    if (!ck(cudaMemsetAsync(counter, 0, sizeof(unsigned) * 4, st), "memset counter")) return false;
    if (!ck(cudaMallocHost(&host_scal, sizeof(double) * 8), "cudaMallocHost")) return false;
    if (!ck(cudaStreamSynchronize(st), "create sync")) return false;
    stats_host = ot_gs_stats();
    return true;
}

// The work decomposition for the given parameters (Sec. 2.3's blocks in
// panels and column chunks) and every device buffer whose size depends on it.
bool Handle::setup_plan(const PlanParams& pp)
{
    if (!plan_allocs.empty()) {
        if (!ck(cudaStreamSynchronize(st), "re-plan sync")) return false;
        free_plan();
        std::vector<const int32_t*> lp(nprob);
        int64_t off = 0;
        for (int32_t k = 0; k < nprob; k++) {
            lp[k] = labels_h.data() + off;
            off += pm_h[k];
        }
        HostPlan nhp;
        std::string pe = build_plan_batch(nprob, lp.data(), pm_h.data(), pn_h.data(), pL_h.data(), pp, nhp);
        if (!pe.empty()) return fail(OTGS_EINVAL, pe);
        hp = std::move(nhp);
    }
    plan_params = pp;
    plan_gen++;
    dp.prows = plan_upload(this, hp.prows, "prows");
    dp.pW = plan_upload(this, hp.pW, "pW");
    dp.pnch = plan_upload(this, hp.pnch, "pnch");
    dp.pitem = plan_upload(this, hp.pitem, "pitem");
    dp.psplit = plan_upload(this, hp.psplit, "psplit");
    dp.gpanel = plan_upload(this, hp.gpanel, "gpanel");
    dp.item_panel = plan_upload(this, hp.item_panel, "item_panel");
    dp.item_chunk = plan_upload(this, hp.item_chunk, "item_chunk");
    dp.exec_order = plan_upload(this, hp.exec_order, "exec_order");
    dp.desc = plan_upload(this, hp.desc, "item descriptors");
    dp.sets = plan_upload(this, hp.sets, "split block sets");
    dp.stage_row0 = plan_upload(this, hp.stage_row0, "stage rows");
    if (!dp.prows || !dp.pW || !dp.pnch || !dp.pitem || !dp.psplit || !dp.gpanel || !dp.item_panel ||
        !dp.item_chunk || !dp.exec_order || !dp.desc || !dp.sets || !dp.stage_row0)
        return false;
    bprob_h.resize(nprob);
    {
        std::vector<int32_t> first(nprob + 1, hp.nitems());
        for (int p = hp.npanels() - 1; p >= 0; p--) first[hp.pprob[p]] = hp.pitem[p];
        for (int32_t k = 0; k < nprob; k++) {
            BProb& b = bprob_h[k];
            b.roff = hp.proff[k];
            b.coff = hp.pcoff[k];
            b.bcoff = hp.pbcoff[k];
            b.m = hp.pm[k];
            b.n = hp.pn[k];
            b.voff = b.roff + b.coff;
            b.item0 = first[k];
            b.item1 = first[k + 1];
        }
    }
    bprob = plan_upload(this, bprob_h, "batch problem table");
    if (!bprob) return false;
    split_part =
        (float*)plan_alloc(sizeof(float) * SPLIT_VALS * ITEM_COLS * (size_t)hp.nsplit_slots, "split partial sums");
    if (!split_part) return false;
    {
        int64_t ce = 0, ct = 0, cc = 0;
        exact_caps(hp, ce, ct, cc);
        if (ce > INT32_MAX || ct > INT32_MAX || cc > INT32_MAX)
            return fail(OTGS_EINVAL, "too many blocks");
        xent_cap = (int32_t)ce;
        xtall_cap = (int32_t)ct;
        xtcol_cap = (int32_t)cc;
        xent = (XEntry*)plan_alloc(sizeof(XEntry) * (size_t)ce, "flagged block sets");
        xtall = (XEntry*)plan_alloc(sizeof(XEntry) * (size_t)ct, "flagged block sets of tall classes");
        xtmap = (uint32_t*)plan_alloc(sizeof(uint32_t) * (size_t)std::max<int64_t>(cc, 1), "column tasks");
        if (!xent || !xtall || !xtmap) return false;
    }
    if (screen_alloc) {
        item_active = (uint8_t*)plan_alloc((size_t)hp.nitems(), "item_active");
        stage_m8 = (uint8_t*)plan_alloc((size_t)hp.nstages * STAGE_ROWS, "stage masks");
        stage_need = (uint32_t*)plan_alloc(sizeof(uint32_t) * (size_t)((hp.nstages + 31) / 32), "stages needed");
        if (!item_active || !stage_m8 || !stage_need) return false;
        invalidate_screen();
    }
    return ck(cudaGetLastError(), "plan upload");
}

EvalArgs Handle::eval_args(const uint8_t* active, const uint32_t* need, bool snap)
{
    EvalArgs e;
    memset(&e, 0, sizeof(e));
    e.probs = probs;
    e.maps = maps;
    if (nprob == 1) {
        e.tm0 = tm0;
        e.pd0 = probs_h[0];
        e.inline_maps = 1;
    }
    e.m = (int32_t)m; e.n = (int32_t)n; e.L = L; e.ntiles = ntiles;
    e.fx_m = (int32_t)hp.max_m; e.fx_n = (int32_t)hp.max_n;
    e.nitems = hp.nitems();
    e.rowA = rowA; e.rowg = dp.rowg;
    e.B2 = B2;
    e.ctl = ctl; e.err = kerr;
    e.nlist = hp.nitems();
    e.desc = dp.desc;
    e.stage_row0 = dp.stage_row0;
    e.item_active = active;
    e.unit_need = need;
    e.unit_words = unit_words;
    e.rowfx = rowfx; e.colfx = colfx;
    // psi goes to the control word (cleared with it) on the single-problem
    // paths; the batch paths point it to their per-problem array
    e.psix = ctl_psi(ctl);
    e.xent = xent; e.xent_cap = xent_cap;
    e.xtall = xtall; e.xtall_cap = xtall_cap;
    e.xtmap = xtmap;
    e.nprob = nprob;
    e.xtcol_cap = xtcol_cap;
    e.fcount = fcount;
    e.use_ct = 1;
    e.wait_ns = (unsigned long long)std::max<int64_t>(dbg_stall_ns, 0);
    e.stall = dbg_stall_ns > 0;
    e.split_part = split_part;
    e.sets = dp.sets; e.nsets = (int32_t)hp.sets.size();
    e.gate = eval_gate;
    e.zt = snap ? zt : nullptr;
    e.ot = snap ? ot : nullptr;
    const double theta = prm.mu * prm.gamma;
    e.theta_hi = (float)theta;
    e.theta_lo = (float)(theta - (double)e.theta_hi);
    double cut = theta * theta * (1.0 - std::ldexp(1.0, -20));
    float fc = (float)cut;
    if ((double)fc > cut) fc = std::nextafter(fc, 0.f);
    e.th2_cut = fc;
    {
        const double t2 = theta * theta * (1.0 - std::ldexp(1.0, -21));
        float ft = (float)t2;
        if ((double)ft > t2) ft = std::nextafter(ft, 0.f);
        e.thr_flag = ft;
    }
    e.gamma = (float)prm.gamma;
    e.inv2g = 1.0 / (2.0 * prm.gamma);
    e.inv2g_hi = (float)e.inv2g;
    e.inv2g_lo = (float)(e.inv2g - (double)e.inv2g_hi);
    return e;
}

ReduceArgs Handle::reduce_args(const uint8_t* active, double* out_caller, double* G_sorted, const double* dir,
                               const double* beta_ptr)
{
    ReduceArgs r;
    memset(&r, 0, sizeof(r));
    r.m = (int32_t)m; r.n = (int32_t)n; r.nitems = hp.nitems();
    r.fx_m = (int32_t)hp.max_m; r.fx_n = (int32_t)hp.max_n;
    r.perm = dp.perm;
    r.item_active = active;
    r.rowfx = rowfx; r.colfx = colfx;
    r.psix = ctl_psi(ctl);
    r.ctl = ctl;
    r.gamma = (float)prm.gamma;
    r.a_sorted = a_sorted; r.b = b;
    r.alpha_sorted = alpha_eval; r.beta = beta_ptr;
    r.out_caller = out_caller; r.G_sorted = G_sorted; r.dir = dir;
    r.scal = scal;
    r.block_part = block_part;
    r.counter = counter;
    r.err = kerr;
    r.gate = eval_gate;
    return r;
}

// Preparation of an evaluation at (alpha, beta); alpha in caller order unless alpha_sorted.
void Handle::prep(const double* alpha, bool alpha_sorted, const double* beta)
{
    launch_prep(alpha, alpha_sorted, dp.perm, beta, (int32_t)m, (int32_t)n, rowA, B2, alpha_eval, rowfx, colfx,
                ctl, st);
}

// Launch of the evaluation kernel, optionally bracketed by timing events.
int Handle::eval_launch(const EvalArgs& e, int n_ctas)
{
    if (timing) {
        while (ev_pool.size() < ev_used + 2) {
            cudaEvent_t ev;
            if (cudaEventCreate(&ev) != cudaSuccess) { timing = false; break; }
            ev_pool.push_back(ev);
        }
    }
    if (timing) cudaEventRecord(ev_pool[ev_used], st);
    launch_stream(e, n_ctas, st);
    if (timing) {
        cudaEventRecord(ev_pool[ev_used + 1], st);
        ev_used += 2;
    }
    launch_split_finish(e, st);
    launch_exact(e, n_sm, st);
    // k_stream, k_split_finish (when a class is split over items), and the
    // exact sums: k_exact_t, or k_exact and k_exact_tall without the transposed copy
    return 1 + (e.nsets > 0 ? 1 : 0) + (e.use_ct ? 1 : 2);
}

// Dense evaluation at (alpha, beta); alpha in caller order unless alpha_sorted.
bool Handle::eval_dense(const double* alpha, bool alpha_sorted, const double* beta, double* out_caller,
                        double* G_sorted, const double* dir, bool snap)
{
    prep(alpha, alpha_sorted, beta);
    if (!eval_gate) stats_host.kernels += 1;
    return eval_dense_core(beta, out_caller, G_sorted, dir, snap);
}

bool Handle::eval_dense_prepped(const double* beta, double* G_sorted, const double* dir)
{
    return eval_dense_core(beta, nullptr, G_sorted, dir, false);
}

bool Handle::eval_dense_core(const double* beta, double* out_caller, double* G_sorted, const double* dir, bool snap)
{
    EvalArgs e = eval_args(nullptr, nullptr, snap);
    const int nk = eval_launch(e, std::min(CTAS_PER_SM * n_sm, hp.nitems()));
    ReduceArgs r = reduce_args(nullptr, out_caller, G_sorted, dir, beta);
    launch_reduce(r, st);
    if (snap && !zt_tiles()) return false;  // z~ is complete: its tile maxima
    if (!eval_gate) {
        count_dense_evals(1);
        stats_host.kernels += nk + 1 + (snap ? 1 : 0);  // and the reduction, the tile maxima
    }
    return ck(cudaGetLastError(), "eval launch");
}

void Handle::count_dense_evals(int64_t k)
{
    stats_host.evals += k;
    stats_host.blocks_total += k * (int64_t)L * n;
    stats_host.units_total += k * (int64_t)L * ntiles;
    dense_units += k * nonempty_units();
    stats_host.units_computed = dense_units;
    dense_cbytes += (double)k * 4.0 * (double)m * (double)n;
    stats_host.c_bytes = dense_cbytes;
}

void Handle::count_screened_evals(int64_t k)
{
    stats_host.evals += k;
    stats_host.blocks_total += k * (int64_t)L * n;
    stats_host.units_total += k * (int64_t)L * ntiles;
}

int64_t Handle::nonempty_units() const
{
    int64_t ne = 0;
    for (int32_t l = 0; l < L; l++) ne += hp.goff[l + 1] > hp.goff[l];
    return ne * ntiles;
}

}  // namespace otgs

// ================================================================== C ABI
#define H_CHECK(h)                                                            \
    do {                                                                      \
        if (!(h)) return OTGS_EINVAL;                                         \
    } while (0)

extern "C" {

static int create_single(ot_gs** out, const float* C, int64_t ldc, const double* a, const double* b,
                         const int32_t* labels, int64_t m, int64_t n, int32_t L, double gamma, double mu, void* stream,
                         bool shard)
{
    g_create_error.clear();
    if (!out) { g_create_error = "h is NULL"; return OTGS_EINVAL; }
    *out = nullptr;
    if (!C || !a || !b || !labels) { g_create_error = "NULL input pointer"; return OTGS_EINVAL; }
    if (m <= 0 || n <= 0 || L <= 0 || ldc < n) { g_create_error = "need m, n, L > 0 and ldc >= n"; return OTGS_EINVAL; }
    if (!(gamma > 0.0) || !std::isfinite(gamma) || !(mu >= 0.0) || !std::isfinite(mu)) {
        g_create_error = "need gamma > 0 and mu >= 0, finite";
        return OTGS_EINVAL;
    }
    Handle* h = new (std::nothrow) Handle();
    if (!h) { g_create_error = "out of host memory"; return OTGS_ENOMEM; }
    h->shard = shard;
    if (!h->init(1, &C, &ldc, &a, &b, &labels, &m, &n, &L, gamma, mu, (cudaStream_t)stream)) {
        g_create_error = h->err;
        int code = h->last_code ? h->last_code : OTGS_ECUDA;
        delete h;
        return code;
    }
    *out = reinterpret_cast<ot_gs*>(h);
    return OTGS_OK;
}

int ot_gs_create(ot_gs** out, const float* C, int64_t ldc, const double* a, const double* b,
                 const int32_t* labels, int64_t m, int64_t n, int32_t L, double gamma, double mu, void* stream)
{
    return create_single(out, C, ldc, a, b, labels, m, n, L, gamma, mu, stream, false);
}

int ot_gs_create_shard(ot_gs** out, const float* C, int64_t ldc, const double* a, const double* b,
                       const int32_t* labels, int64_t m, int64_t n, int32_t L, double gamma, double mu, void* stream)
{
    return create_single(out, C, ldc, a, b, labels, m, n, L, gamma, mu, stream, true);
}

int ot_gs_destroy(ot_gs* hh)
{
    if (!hh) return OTGS_OK;
    delete reinterpret_cast<Handle*>(hh);
    return OTGS_OK;
}

int ot_gs_set_stream(ot_gs* hh, void* stream)
{
    H_CHECK(hh);
    reinterpret_cast<Handle*>(hh)->st = (cudaStream_t)stream;
    return OTGS_OK;
}

int ot_gs_set_params(ot_gs* hh, const ot_gs_params* p)
{
    H_CHECK(hh);
    Handle* h = reinterpret_cast<Handle*>(hh);
    if (!p) { h->fail(OTGS_EINVAL, "params is NULL"); return OTGS_EINVAL; }
    if (!(p->gamma > 0.0) || !std::isfinite(p->gamma) || !(p->mu >= 0.0) || !std::isfinite(p->mu) || p->r < 1 ||
        p->lbfgs_m < 1 || p->lbfgs_m > 32 || !(p->ftol >= 0.0)) {
        h->fail(OTGS_EINVAL, "invalid params (gamma > 0, mu >= 0, r >= 1, 1 <= lbfgs_m <= 32, ftol >= 0)");
        return OTGS_EINVAL;
    }
    bool reg_changed = p->gamma != h->prm.gamma || p->mu != h->prm.mu;
    h->prm = *p;
    if (reg_changed) h->invalidate_screen();
    return OTGS_OK;
}

int ot_gs_get_params(const ot_gs* hh, ot_gs_params* p)
{
    H_CHECK(hh);
    if (!p) return OTGS_EINVAL;
    *p = reinterpret_cast<const Handle*>(hh)->prm;
    return OTGS_OK;
}

int ot_gs_grad(ot_gs* hh, const double* alpha, const double* beta, double* out)
{
    H_CHECK(hh);
    Handle* h = reinterpret_cast<Handle*>(hh);
    if (!single_problem(h)) return OTGS_EINVAL;
    if (!alpha || !beta || !out) { h->fail(OTGS_EINVAL, "NULL pointer"); return OTGS_EINVAL; }
    if (!h->eval_dense(alpha, false, beta, out, nullptr, nullptr, false)) return h->last_code;
    return OTGS_OK;
}

int ot_gs_get_stats(ot_gs* hh, ot_gs_stats* s)
{
    H_CHECK(hh);
    Handle* h = reinterpret_cast<Handle*>(hh);
    if (!s) return OTGS_EINVAL;
    if (!h->ck(cudaStreamSynchronize(h->st), "stats sync")) return OTGS_ECUDA;
    if (!h->collect_stats()) return h->last_code;
    unsigned long long fc[2] = {0, 0};
    if (!h->ck(cudaMemcpy(fc, h->fcount, sizeof(fc), cudaMemcpyDeviceToHost), "stats D2H")) return OTGS_ECUDA;
    h->stats_host.blocks_flagged = (int64_t)fc[0];
    *s = h->stats_host;
    return OTGS_OK;
}

int ot_gs_reset_stats(ot_gs* hh)
{
    H_CHECK(hh);
    Handle* h = reinterpret_cast<Handle*>(hh);
    if (!h->ck(cudaStreamSynchronize(h->st), "stats sync")) return OTGS_ECUDA;
    h->stats_host = ot_gs_stats();
    h->reset_device_stats();
    if (!h->ck(cudaMemsetAsync(h->fcount, 0, sizeof(unsigned long long) * 2, h->st), "memset counters"))
        return OTGS_ECUDA;
    return OTGS_OK;
}

int ot_gs_debug(ot_gs* hh, int what, int64_t value)
{
    H_CHECK(hh);
    Handle* h = reinterpret_cast<Handle*>(hh);
    if (what == OTGS_DEBUG_STALL) {
        if (value > 10000000000LL) {
            h->fail(OTGS_EINVAL, "stall wait limit above 10 s");
            return OTGS_EINVAL;
        }
        h->dbg_stall_ns = value > 0 ? value : 0;
        return OTGS_OK;
    }
    if (what == OTGS_DEBUG_SCREEN_ROUTE) {
        if (value < 0 || value > 2) {
            h->fail(OTGS_EINVAL, "screen route is 0, 1 or 2");
            return OTGS_EINVAL;
        }
        h->dbg_route = value;
        return OTGS_OK;
    }
    if (what == OTGS_DEBUG_NAN_EVAL) {
        h->dbg_nan_eval = value > 0 ? value : 0;
        return OTGS_OK;
    }
    h->fail(OTGS_EINVAL, "unknown debug switch");
    return OTGS_EINVAL;
}

int ot_gs_set_timing(ot_gs* hh, int enable)
{
    H_CHECK(hh);
    Handle* h = reinterpret_cast<Handle*>(hh);
    h->timing = enable != 0;
    return OTGS_OK;
}

int ot_gs_get_timing(ot_gs* hh, int64_t* launches, double* total_ms)
{
    H_CHECK(hh);
    Handle* h = reinterpret_cast<Handle*>(hh);
    if (!h->ck(cudaStreamSynchronize(h->st), "timing sync")) return OTGS_ECUDA;
    double tot = 0.0;
    for (size_t k = 0; k + 1 < h->ev_used; k += 2) {
        float ms = 0.f;
        if (!h->ck(cudaEventElapsedTime(&ms, h->ev_pool[k], h->ev_pool[k + 1]), "cudaEventElapsedTime"))
            return OTGS_ECUDA;
        tot += ms;
    }
    if (launches) *launches = (int64_t)(h->ev_used / 2);
    if (total_ms) *total_ms = tot;
    h->ev_used = 0;
    return OTGS_OK;
}

const char* ot_gs_last_error(const ot_gs* hh)
{
    if (!hh) return g_create_error.c_str();
    return reinterpret_cast<const Handle*>(hh)->err.c_str();
}

const char* ot_gs_version(void) { return "otgs 0.1 sm_103a"; }

int ot_gs_plan_info(const int32_t* labels_host, int64_t m, int64_t n, int32_t L, int64_t* n_panels,
                    int64_t* n_items, int64_t* n_stages)
{
    if (!labels_host) return OTGS_EINVAL;
    HostPlan hp;
    if (!build_plan(labels_host, m, n, L, hp).empty()) return OTGS_EINVAL;
    if (n_panels) *n_panels = hp.npanels();
    if (n_items) *n_items = hp.nitems();
    if (n_stages) *n_stages = hp.nstages;
    return OTGS_OK;
}

int ot_gs_plan_info_batch(int32_t nprob, const int32_t* const* labels_host, const int64_t* m, const int64_t* n,
                          const int32_t* L, int32_t panel_rows, int32_t split_rows, int32_t stage_fill,
                          int64_t* n_panels, int64_t* n_items, int64_t* n_stages)
{
    if (nprob <= 0 || !labels_host || !m || !n || !L || panel_rows < 0 || split_rows < 0 || stage_fill < 0 ||
        stage_fill > STAGE_ROWS)
        return OTGS_EINVAL;
    HostPlan hp;
    PlanParams pp;
    pp.panel_rows = panel_rows;
    pp.split_rows = split_rows;
    pp.stage_fill = stage_fill;
    if (!build_plan_batch(nprob, labels_host, m, n, L, pp, hp).empty()) return OTGS_EINVAL;
    if (n_panels) *n_panels = hp.npanels();
    if (n_items) *n_items = hp.nitems();
    if (n_stages) *n_stages = hp.nstages;
    return OTGS_OK;
}

}  // extern "C"
