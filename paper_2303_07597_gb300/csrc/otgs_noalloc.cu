// otgs_noalloc.cu -- a dense evaluation that allocates no device memory.
//
// ot_gs_grad needs a handle, and creating one allocates device buffers.  Some
// callers cannot do that: code that runs inside a custom device allocator's
// callbacks (cudaMalloc there would recurse or deadlock), frameworks whose
// memory pool forbids allocations outside the pool, and latency-critical loops
// that cannot afford cudaMalloc's implicit device synchronisation.  This entry
// point serves them: every scratch buffer of the evaluation -- the group plan,
// the float-pair split of alpha and beta and its bounds, the row / column / psi
// partial sums, the work counter, the error word and the reduction's block
// partials -- is carved out of one file-scope
// __device__ array of OTGS_STATIC_SCRATCH_BYTES bytes.  Each GPU that loads
// this part of the library keeps that array until the process exits.
//
// In host code the array's name is only a host-side stand-in for the symbol,
// not a device address.  Its device address is looked up once per device with
// cudaGetSymbolAddress, with that device current, on the first call made
// while that device is current; that first call should therefore come before
// any stream capture.  All calls share the array and it keeps the contents of
// the last call: the values that must start at zero (the reduction's ticket
// counter, the evaluation's work counter and error word) are cleared by every
// call.  Calls that overlap on the GPU (on
// different streams, or from different host threads) race on the array.
#include <cmath>
#include <cstring>
#include <mutex>
#include <string>
#include <vector>

#include "otgs_internal.cuh"

namespace otgs {

static __device__ __align__(256) unsigned char g_static_scratch[OTGS_STATIC_SCRATCH_BYTES];

namespace {

constexpr int kMaxDevices = 128;
std::mutex g_mu;
void* g_addr[kMaxDevices] = {nullptr};
thread_local std::string g_err;

int set_err(int code, const std::string& msg)
{
    g_err = msg;
    return code;
}

// Bump allocator over the static array (offsets only; no memory is allocated).
struct Carve {
    size_t off = 0;
    size_t take(size_t bytes)
    {
        size_t at = (off + 255) / 256 * 256;
        off = at + (bytes ? bytes : 1);
        return at;
    }
};

}  // namespace

}  // namespace otgs

using namespace otgs;

extern "C" {

const char* ot_gs_noalloc_last_error(void) { return g_err.c_str(); }

int ot_gs_grad_noalloc(const float* C, int64_t ldc, const double* a, const double* b, const int32_t* labels_host,
                       int64_t m, int64_t n, int32_t L, double gamma, double mu, const double* alpha,
                       const double* beta, double* out, void* stream)
{
    g_err.clear();
    if (!C || !a || !b || !labels_host || !alpha || !beta || !out)
        return set_err(OTGS_EINVAL, "NULL pointer");
    if (m <= 0 || n <= 0 || L <= 0 || ldc < n) return set_err(OTGS_EINVAL, "need m, n, L > 0 and ldc >= n");
    if (!(gamma > 0.0) || !std::isfinite(gamma) || !(mu >= 0.0) || !std::isfinite(mu))
        return set_err(OTGS_EINVAL, "need gamma > 0 and mu >= 0, finite");
    if (ldc % 4 != 0 || reinterpret_cast<uintptr_t>(C) % 16 != 0)
        return set_err(OTGS_EINVAL, "need ldc % 4 == 0 and a 16-byte aligned C");
    for (int64_t i = 1; i < m; i++)
        if (labels_host[i] < labels_host[i - 1])
            return set_err(OTGS_EINVAL, "labels must be non-decreasing (class-sorted rows of C)");
    HostPlan hp;
    std::string pe = build_plan(labels_host, m, n, L, hp);
    if (!pe.empty()) return set_err(OTGS_EINVAL, pe);
    const int ntiles = hp.ntiles;
    // layout of the scratch array
    Carve cv;
    const size_t o_perm = cv.take(4 * hp.perm.size()), o_rowg = cv.take(sizeof(int4) * hp.rowg.size());
    const size_t o_desc = cv.take(sizeof(ItemDesc) * hp.desc.size());
    const size_t o_st = cv.take(sizeof(int32_t) * hp.stage_row0.size());
    const size_t o_rowA = cv.take(sizeof(float4) * (size_t)m);
    const size_t o_B2 = cv.take(8 * (size_t)padded_cols(n));
    const size_t o_ctl = cv.take(sizeof(EvalCtl)), o_err = cv.take(16);
    const size_t o_aeval = cv.take(8 * (size_t)m);
    const size_t o_rowfx = cv.take(8 * (size_t)m), o_colfx = cv.take(8 * (size_t)n);
    const size_t o_spart = cv.take(sizeof(float) * SPLIT_VALS * ITEM_COLS * (size_t)hp.nsplit_slots);
    int64_t xe_cap = 0, xt_cap = 0;
    int64_t xc_cap = 0;  // (the transposed route's; not used here)
    exact_caps(hp, xe_cap, xt_cap, xc_cap);
    const size_t o_xent = cv.take(sizeof(XEntry) * (size_t)xe_cap);
    const size_t o_xtall = cv.take(sizeof(XEntry) * (size_t)xt_cap);
    const size_t o_sets = cv.take(sizeof(SplitSet) * hp.sets.size());
    const size_t o_maps = cv.take(sizeof(TmaMaps)), o_prob = cv.take(sizeof(ProbDesc));
    const int nred = reduce_blocks((int32_t)m, (int32_t)n);
    const size_t o_bpart = cv.take(8 * REDUCE_PARTS * (size_t)nred), o_counter = cv.take(16), o_scal = cv.take(64);
    if (cv.off > OTGS_STATIC_SCRATCH_BYTES)
        return set_err(OTGS_EINVAL, "problem needs " + std::to_string(cv.off) + " bytes of scratch, above the " +
                                        std::to_string((size_t)OTGS_STATIC_SCRATCH_BYTES) +
                                        " bytes of the static buffer");
    // per-device set-up: the device address of the static array
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return set_err(OTGS_ECUDA, std::string("cudaGetDevice: ") + cudaGetErrorString(e));
    if (dev < 0 || dev >= kMaxDevices) return set_err(OTGS_EINVAL, "device index out of range");
    unsigned char* base = nullptr;
    {
        std::lock_guard<std::mutex> lk(g_mu);
        if (!g_addr[dev]) {
            void* p = nullptr;
            e = cudaGetSymbolAddress(&p, g_static_scratch);
            if (e != cudaSuccess || !p)
                return set_err(OTGS_ECUDA, std::string("cudaGetSymbolAddress: ") + cudaGetErrorString(e));
            g_addr[dev] = p;
        }
        base = static_cast<unsigned char*>(g_addr[dev]);
    }
    cudaStream_t st = (cudaStream_t)stream;
    auto up = [&](size_t off, const void* src, size_t bytes) {
        return bytes == 0 ? cudaSuccess : cudaMemcpyAsync(base + off, src, bytes, cudaMemcpyHostToDevice, st);
    };
    e = up(o_perm, hp.perm.data(), 4 * hp.perm.size());
    if (e == cudaSuccess) e = up(o_rowg, hp.rowg.data(), sizeof(int4) * hp.rowg.size());
    if (e == cudaSuccess) e = up(o_desc, hp.desc.data(), sizeof(ItemDesc) * hp.desc.size());
    if (e == cudaSuccess) e = up(o_st, hp.stage_row0.data(), sizeof(int32_t) * hp.stage_row0.size());
    if (e == cudaSuccess) e = cudaMemsetAsync(base + o_counter, 0, 16, st);
    if (e == cudaSuccess) e = cudaMemsetAsync(base + o_err, 0, 16, st);
    if (e == cudaSuccess) e = up(o_sets, hp.sets.data(), sizeof(SplitSet) * hp.sets.size());
    TmaMaps tm;
    {
        const std::string te = make_tmaps(C, ldc, m, n, tm);
        if (!te.empty()) return set_err(OTGS_ECUDA, te);
    }
    ProbDesc pd;
    memset(&pd, 0, sizeof(pd));
    pd.C = C; pd.ldc = ldc; pd.m = (int32_t)m; pd.n = (int32_t)n;
    if (e == cudaSuccess) e = up(o_maps, &tm, sizeof(tm));
    if (e == cudaSuccess) e = up(o_prob, &pd, sizeof(pd));
    int n_sm = 0;
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&n_sm, cudaDevAttrMultiProcessorCount, dev);
    if (e != cudaSuccess) return set_err(OTGS_ECUDA, std::string("scratch upload: ") + cudaGetErrorString(e));
    const int32_t* perm = (const int32_t*)(base + o_perm);
    float4* rowA = (float4*)(base + o_rowA);
    float2* B2 = (float2*)(base + o_B2);
    EvalCtl* ctl = (EvalCtl*)(base + o_ctl);
    double* aeval = (double*)(base + o_aeval);
    unsigned long long* rowfx = (unsigned long long*)(base + o_rowfx);
    unsigned long long* colfx = (unsigned long long*)(base + o_colfx);
    // the caller's alpha is already in class-sorted order (labels non-decreasing)
    launch_prep(alpha, true, perm, beta, (int32_t)m, (int32_t)n, rowA, B2, aeval, rowfx, colfx, ctl, st);
    EvalArgs ea;
    memset(&ea, 0, sizeof(ea));
    ea.probs = (const ProbDesc*)(base + o_prob);
    ea.maps = (const CUtensorMap*)(base + o_maps);
    ea.tm0 = tm;
    ea.pd0 = pd;
    ea.inline_maps = 1;
    ea.m = (int32_t)m; ea.n = (int32_t)n; ea.L = L; ea.ntiles = ntiles;
    ea.fx_m = (int32_t)m; ea.fx_n = (int32_t)n;
    ea.nitems = hp.nitems();
    ea.rowA = rowA; ea.rowg = (const int4*)(base + o_rowg);
    ea.B2 = B2;
    ea.ctl = ctl; ea.err = (int*)(base + o_err);
    ea.nlist = hp.nitems();
    ea.desc = (const ItemDesc*)(base + o_desc);
    ea.stage_row0 = (const int32_t*)(base + o_st);
    ea.item_active = nullptr; ea.unit_need = nullptr;
    ea.unit_words = (ntiles + 31) / 32;
    ea.rowfx = rowfx; ea.colfx = colfx;
    ea.psix = ctl_psi(ctl);  // cleared with the control word by the preparation
    ea.xent = (XEntry*)(base + o_xent);
    ea.xent_cap = (int32_t)xe_cap;
    ea.xtall = (XEntry*)(base + o_xtall);
    ea.xtall_cap = (int32_t)xt_cap;
    ea.split_part = (float*)(base + o_spart);
    ea.sets = (const SplitSet*)(base + o_sets);
    ea.nsets = (int32_t)hp.sets.size();
    const double theta = mu * gamma;
    ea.theta_hi = (float)theta;
    ea.theta_lo = (float)(theta - (double)ea.theta_hi);
    const double cut = theta * theta * (1.0 - std::ldexp(1.0, -20));
    float fc = (float)cut;
    if ((double)fc > cut) fc = std::nextafter(fc, 0.f);
    ea.th2_cut = fc;
    {
        const double t2 = theta * theta * (1.0 - std::ldexp(1.0, -21));
        float ft = (float)t2;
        if ((double)ft > t2) ft = std::nextafter(ft, 0.f);
        ea.thr_flag = ft;
    }
    ea.gamma = (float)gamma;
    ea.inv2g = 1.0 / (2.0 * gamma);
    ea.inv2g_hi = (float)ea.inv2g;
    ea.inv2g_lo = (float)(ea.inv2g - (double)ea.inv2g_hi);
    if (!stream_prepare()) return set_err(OTGS_ECUDA, "cudaFuncSetAttribute(evaluation kernel)");
    launch_stream(ea, std::min(CTAS_PER_SM * n_sm, hp.nitems()), st);
    launch_split_finish(ea, st);
    launch_exact(ea, n_sm, st);
    ReduceArgs ra;
    memset(&ra, 0, sizeof(ra));
    ra.m = (int32_t)m; ra.n = (int32_t)n; ra.nitems = hp.nitems();
    ra.fx_m = (int32_t)m; ra.fx_n = (int32_t)n;
    ra.perm = perm; ra.item_active = nullptr;
    ra.rowfx = rowfx; ra.colfx = colfx; ra.psix = ea.psix;
    ra.ctl = ctl; ra.gamma = ea.gamma;
    ra.a_sorted = a; ra.b = b; ra.alpha_sorted = aeval; ra.beta = beta;
    ra.out_caller = out; ra.scal = (double*)(base + o_scal);
    ra.block_part = (double*)(base + o_bpart);
    ra.counter = (unsigned*)(base + o_counter);
    ra.err = ea.err;
    launch_reduce(ra, st);
    e = cudaGetLastError();
    if (e != cudaSuccess) return set_err(OTGS_ECUDA, std::string("launch: ") + cudaGetErrorString(e));
    return OTGS_OK;
}

}  // extern "C"
