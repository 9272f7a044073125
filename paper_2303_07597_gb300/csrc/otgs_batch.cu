// otgs_batch.cu -- many independent problems in one handle: one evaluation
// kernel streams every problem's C (the block-diagonal plan of otgs_plan.cu),
// and the per-problem work (preparation, the reduction to D and its
// gradient, the L-BFGS step) runs one CTA per problem.
//
// The batched solver keeps a separate L-BFGS state per problem (its own
// memory, line search and stopping test), so each problem follows the same
// iteration as a solve on its own; only the evaluations are shared.  One
// trial is five kernels:
//   k_bgate        opens the trial when some problem is still running,
//   k_stream       the evaluation of every running problem (finished
//                  problems' work items are skipped),
//   k_split_finish, k_exact   as for one problem,
//   k_bstep        per problem: the reduction to D, Gt.d and ||Gt||_inf, the
//                  line-search step, on acceptance the L-BFGS update and the
//                  new direction (the recursion of Nocedal & Wright, Alg. 7.4),
//                  and the preparation of the next trial point.
// The host captures a fixed number of trials in a CUDA graph and relaunches
// it until every problem has stopped.
#include <algorithm>
#include <cmath>
#include <cstring>

#include "otgs_solver.cuh"

namespace otgs {

#define FULLMASK 0xffffffffu

constexpr int BT = 512;                // threads of the per-problem kernels
constexpr int BW = BT / 32;
constexpr int TRIALS_PER_GRAPH = 16;   // trials captured in one graph

enum { PH_START = 0, PH_LS = 1 };

// Per-problem L-BFGS state (the fields the shared line-search and direction
// steps use, plus the batch's own).
struct BState {
    int status, done, iter, npairs, head, ls_evals, have_hi, force_accept, phase, pad;
    long long evals;
    double t, lo, Flo, dlo, hi, Fhi, dhi;
    double F, F0, dphi0, ginf, cG;
    double target;     // stop when D >= target - rtol |target| (NaN: no target)
    double t_done_ms;  // device time from the start of the solve to the stop
    double SY[MAX_LBFGS_M * MAX_LBFGS_M];
    double YY[MAX_LBFGS_M * MAX_LBFGS_M];
    double cy[MAX_LBFGS_M], cs[MAX_LBFGS_M];
};

struct BCtl {
    int nactive;  // problems still running
    int go;       // the current trial runs
    unsigned long long t_begin;
};

struct BResult {
    int status, iter;
    long long evals;
    double D, ginf, t_ms;
};

struct BStepArgs {
    const BProb* P;
    BState* S;
    BCtl* bc;
    int* pactive;
    FxScale* pfx;    // per problem: the fixed-point scale of its evaluation point
    float gamma;
    unsigned long long* rowfx;
    unsigned long long* colfx;
    unsigned long long* psix;        // [nprob][2]: psi of the problem's flagged blocks, fixed point
    const int* kerr;
    const double* a_sorted;
    const double* b;
    double *x, *G, *d, *xt, *Gt;
    float2 *Sv, *Yv;  // history s_k, y_k as float pairs (hi, lo), slot-major
    float2* Gp;       // the current G as float pairs
    int64_t Ntot;
    int M;
    float4* rowA;
    float2* B2;
    double tol, rtol, ftol;
    int maxit;
};

struct Batch {
    Handle* h = nullptr;
    int nprob = 0, M = 0;
    int64_t Ntot = 0;
    BState* S = nullptr;
    BCtl* bc = nullptr;
    BCtl* hbc = nullptr;  // pinned: two slots of nactive read-backs
    int* pactive = nullptr;
    double *x = nullptr, *G = nullptr, *d = nullptr, *xt = nullptr, *Gt = nullptr;
    float2 *Sv = nullptr, *Yv = nullptr, *Gp = nullptr;
    BResult* res = nullptr;
    cudaStream_t bst = nullptr;
    cudaEvent_t ev[3] = {nullptr, nullptr, nullptr};
    cudaGraphExec_t gexec = nullptr;
    int g_plan = -1;  // generation of the plan the graph was captured with
    double g_tol = -1.0, g_rtol = -1.0, g_ftol = -1.0;
    double g_gamma = -1.0, g_mu = -1.0;  // regularisation baked into the captured kernels' arguments
    int g_maxit = -1;
    ~Batch();
};

void destroy_batch(Batch* b) { delete b; }

Batch::~Batch()
{
    if (bst) cudaStreamSynchronize(bst);
    if (gexec) cudaGraphExecDestroy(gexec);
    for (cudaEvent_t e : ev)
        if (e) cudaEventDestroy(e);
    if (bst) cudaStreamDestroy(bst);
    if (hbc) cudaFreeHost(hbc);
}

__device__ __forceinline__ unsigned long long b_gtimer()
{
    unsigned long long t;
    asm volatile("mov.u64 %0, %globaltimer;" : "=l"(t));
    return t;
}

// Fixed-order CTA sums of NV values per thread; every thread gets the totals.
template <int NV>
__device__ __forceinline__ void cta_sum(double (&v)[NV], double* sh /* [BW * NV] */, double* out /* [NV] */)
{
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
#pragma unroll
    for (int k = 0; k < NV; k++) {
        double x = v[k];
#pragma unroll
        for (int off = 16; off >= 1; off >>= 1) x += __shfl_xor_sync(FULLMASK, x, off);
        if (lane == 0) sh[w * NV + k] = x;
    }
    __syncthreads();
    if (threadIdx.x < NV) {
        double s = 0.0;
        for (int q = 0; q < BW; q++) s += sh[q * NV + threadIdx.x];
        out[threadIdx.x] = s;
    }
    __syncthreads();
#pragma unroll
    for (int k = 0; k < NV; k++) v[k] = out[k];
}

// The same for integers (exact: the order of the additions does not matter).
template <int NV>
__device__ __forceinline__ void cta_sum_ll(long long (&v)[NV], long long* sh /* [BW * NV] */, long long* out)
{
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
#pragma unroll
    for (int k = 0; k < NV; k++) {
        long long x = v[k];
#pragma unroll
        for (int off = 16; off >= 1; off >>= 1) x += __shfl_xor_sync(FULLMASK, x, off);
        if (lane == 0) sh[w * NV + k] = x;
    }
    __syncthreads();
    if (threadIdx.x < NV) {
        long long s = 0;
        for (int q = 0; q < BW; q++) s += sh[q * NV + threadIdx.x];
        out[threadIdx.x] = s;
    }
    __syncthreads();
#pragma unroll
    for (int k = 0; k < NV; k++) v[k] = out[k];
}

__device__ __forceinline__ double cta_max(double v, double* sh /* [BW] */)
{
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
#pragma unroll
    for (int off = 16; off >= 1; off >>= 1) v = fmax(v, __shfl_xor_sync(FULLMASK, v, off));
    if (lane == 0) sh[w] = v;
    __syncthreads();
    double r = 0.0;
    for (int q = 0; q < BW; q++) r = fmax(r, sh[q]);
    __syncthreads();
    return r;
}

// The problem's maxima [alpha hi]_+, [beta hi]_+ (non-negative floats
// compare as their bits) and the fixed-point scale they give, for the
// problem's next evaluation; all threads call it.
__device__ __forceinline__ void store_scale(float apos, float bpos, int k, const BProb& p, float gamma,
                                            FxScale* pfx, unsigned* sh /* [2 * BW] */)
{
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const unsigned ma = __reduce_max_sync(FULLMASK, __float_as_uint(apos));
    const unsigned mb = __reduce_max_sync(FULLMASK, __float_as_uint(bpos));
    if (lane == 0) {
        sh[w] = ma;
        sh[BW + w] = mb;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        unsigned ua = 0u, ub = 0u;
        for (int q = 0; q < BW; q++) {
            ua = max(ua, sh[q]);
            ub = max(ub, sh[BW + q]);
        }
        pfx[k] = fx_scale(ua, ub, p.m, p.n, gamma);
    }
}

// --------------------------------------------------- evaluation (C ABI)
// Preparation of one problem per CTA from the caller's concatenated alpha
// (caller row order within a problem) and beta.
__global__ void __launch_bounds__(BT) k_bprep(const BProb* __restrict__ P, const double* __restrict__ alpha,
                                              const int32_t* __restrict__ perm, const double* __restrict__ beta,
                                              float4* rowA, float2* B2, double* alpha_eval, unsigned long long* rowfx,
                                              unsigned long long* colfx, FxScale* pfx, float gamma,
                                              unsigned long long* psix)
{
    __shared__ unsigned shm[2 * BW];
    const BProb p = P[blockIdx.x];
    if (threadIdx.x < 2) psix[2 * blockIdx.x + threadIdx.x] = 0ull;
    float apos = 0.f, bpos = 0.f;
    for (int e = threadIdx.x; e < p.m; e += BT) {
        const int r = p.roff + e;
        const double a = alpha[perm[r]];
        apos = fmaxf(apos, prep_row(a, rowA + r));
        alpha_eval[r] = a;
        rowfx[r] = 0ull;
    }
    for (int j = threadIdx.x; j < p.n; j += BT) {
        bpos = fmaxf(bpos, prep_col(true, beta[p.coff + j], B2 + p.bcoff + j));
        colfx[p.coff + j] = 0ull;
    }
    store_scale(apos, bpos, blockIdx.x, p, gamma, pfx, shm);
}

// D of each problem and the gradient in the caller's layout.
__global__ void __launch_bounds__(BT) k_breduce(const BProb* __restrict__ P, const int32_t* __restrict__ perm,
                                                const FxScale* pfx,
                                                const unsigned long long* __restrict__ rowfx,
                                                const unsigned long long* __restrict__ colfx,
                                                const unsigned long long* __restrict__ psix, const int* kerr,
                                                const double* __restrict__ a_sorted, const double* __restrict__ b,
                                                const double* __restrict__ alpha_eval,
                                                const double* __restrict__ beta, int64_t m_tot, double* Dout,
                                                double* grad)
{
    __shared__ double sh[BW * 2], tot[2];
    const BProb p = P[blockIdx.x];
    const FxScale fx = pfx[blockIdx.x];
    double v[1] = {0.0};  // alpha.a + beta.b
    for (int e = threadIdx.x; e < p.m; e += BT) {
        const int r = p.roff + e;
        const double ga = a_sorted[r] - (double)(long long)rowfx[r] * fx.from_r;
        if (grad) grad[perm[r]] = ga;
        v[0] += alpha_eval[r] * a_sorted[r];
    }
    for (int j = threadIdx.x; j < p.n; j += BT) {
        const int c = p.coff + j;
        const double gb = b[c] - (double)(long long)colfx[c] * fx.from_c;
        if (grad) grad[m_tot + c] = gb;
        v[0] += beta[c] * b[c];
    }
    cta_sum<1>(v, sh, tot);
    if (threadIdx.x == 0 && Dout) {
        const double psi = psi_from_fx((long long)psix[2 * blockIdx.x], (long long)psix[2 * blockIdx.x + 1], fx.from_p);
        Dout[blockIdx.x] = (kerr && *(volatile const int*)kerr) ? __longlong_as_double(0x7ff8000000000000ll)
                                                                 : v[0] - psi;
    }
}

bool Handle::eval_batch(const double* alpha, const double* beta, double* D, double* grad)
{
    if (!ck(cudaMemsetAsync(ctl, 0, sizeof(EvalCtl), st), "memset")) return false;
    k_bprep<<<nprob, BT, 0, st>>>(bprob, alpha, dp.perm, beta, rowA, B2, alpha_eval, rowfx, colfx, pfx,
                                  (float)prm.gamma, psix);
    EvalArgs e = eval_args(nullptr, nullptr, false);
    e.gate = nullptr;
    e.pfx = pfx;
    e.psix = psix;  // per problem (k_breduce reads them), even for a batch of one
    eval_launch(e, std::min(CTAS_PER_SM * n_sm, hp.nitems()));
    k_breduce<<<nprob, BT, 0, st>>>(bprob, dp.perm, pfx, rowfx, colfx, psix, kerr, a_sorted, b, alpha_eval,
                                    beta, m, D, grad);
    count_dense_evals(1);
    return ck(cudaGetLastError(), "batch evaluation launch");
}

// ------------------------------------------------------ batched solver
__global__ void __launch_bounds__(BT) k_binit(const BProb* __restrict__ P, BState* S, int* pactive, const double* x,
                                              double* xt, float4* rowA, float2* B2, unsigned long long* rowfx,
                                              unsigned long long* colfx, FxScale* pfx, float gamma, int M,
                                              const double* target, unsigned long long* psix)
{
    if (threadIdx.x < 2) psix[2 * blockIdx.x + threadIdx.x] = 0ull;
    __shared__ unsigned shm[2 * BW];
    const int k = blockIdx.x;
    const BProb p = P[k];
    BState* s = S + k;
    if (threadIdx.x == 0) {
        s->status = OTGS_ENOTCONV;
        s->done = 0;
        s->iter = 0;
        s->npairs = 0;
        s->head = 0;
        s->ls_evals = 0;
        s->have_hi = 0;
        s->force_accept = 0;
        s->phase = PH_START;
        s->evals = 0;
        s->t = 0.0;
        s->target = target ? target[k] : __longlong_as_double(0x7ff8000000000000ll);
        s->t_done_ms = 0.0;
        pactive[k] = 1;
    }
    for (int q = threadIdx.x; q < M * M; q += blockDim.x) {
        s->SY[q] = 0.0;
        s->YY[q] = 0.0;
    }
    for (int q = threadIdx.x; q < MAX_LBFGS_M; q += blockDim.x) {
        s->cy[q] = 0.0;
        s->cs[q] = 0.0;
    }
    const double* xv = x + p.voff;
    double* tv = xt + p.voff;
    float apos = 0.f, bpos = 0.f;
    for (int e = threadIdx.x; e < p.m + p.n; e += blockDim.x) {
        const double v = xv[e];
        tv[e] = v;
        if (e < p.m) {
            apos = fmaxf(apos, prep_row(v, rowA + p.roff + e));
            rowfx[p.roff + e] = 0ull;
        } else {
            bpos = fmaxf(bpos, prep_col(true, v, B2 + p.bcoff + (e - p.m)));
            colfx[p.coff + (e - p.m)] = 0ull;
        }
    }
    store_scale(apos, bpos, k, p, gamma, pfx, shm);
}

__global__ void k_bbegin(BCtl* bc) { bc->t_begin = b_gtimer(); }

// Opens a trial while some problem runs (with a cleared control word).
__global__ void k_bgate(BCtl* bc, EvalCtl* ctl)
{
    const int go = bc->nactive > 0;
    bc->go = go;
    if (!go) return;
    ctl_clear(ctl);
}

__device__ __forceinline__ bool reached(const BState* s, double D, double rtol)
{
    return s->target == s->target && D >= s->target - rtol * fabs(s->target);
}

enum { ACT_RETRY = 0, ACT_ACCEPT = 1, ACT_START = 2 };

constexpr int SLOT_GROUP = 4;  // history slots whose dot products one pass accumulates

// Double-float arithmetic for the history's dot products and combinations:
// FP64 runs at a small fraction of FP32's rate on GB300, and these are most
// of a solver step's work.  A float pair (hi, lo) holds an FP64 value to
// ~2^-48 relative; the product of two pairs and a running sum keep that
// accuracy (Dekker's product by FMA, Knuth's TwoSum), so a dot of n terms is
// within ~n 2^-48 of its FP64 value.
__device__ __forceinline__ float2 dsplit(double x)
{
    const float h = __double2float_rn(x);
    return make_float2(h, __double2float_rn(x - (double)h));
}

// (h, l) += a * b
__device__ __forceinline__ void dd_fma(float2 a, float2 b, float& h, float& l)
{
    const float p = __fmul_rn(a.x, b.x);
    float e = fmaf(a.x, b.x, -p);
    e = fmaf(a.x, b.y, fmaf(a.y, b.x, e));
    const float s = __fadd_rn(h, p);
    const float bb = __fsub_rn(s, h);
    const float err = __fadd_rn(__fsub_rn(h, __fsub_rn(s, bb)), __fsub_rn(p, bb));
    h = s;
    l = __fadd_rn(l, __fadd_rn(err, e));
}

__device__ __forceinline__ double dd_value(float h, float l) { return (double)h + (double)l; }

// Warp sums of NV double-float values (a fixed xor tree, in FP32 pairs: an
// FP64 tree of these would be most of the step's FP64 work); lane 0 writes
// the totals, as FP64, to dst.
template <int NV>
__device__ __forceinline__ void warp_dd_sums_to(float (&h)[NV], float (&l)[NV], double* dst)
{
#pragma unroll
    for (int c = 0; c < NV; c++) {
        float hh = h[c], ll = l[c];
#pragma unroll
        for (int off = 16; off >= 1; off >>= 1) {
            const float oh = __shfl_xor_sync(FULLMASK, hh, off), ol = __shfl_xor_sync(FULLMASK, ll, off);
            const float s = __fadd_rn(hh, oh);
            const float bb = __fsub_rn(s, hh);
            const float err = __fadd_rn(__fsub_rn(hh, __fsub_rn(s, bb)), __fsub_rn(oh, bb));
            hh = s;
            ll = __fadd_rn(__fadd_rn(ll, ol), err);
        }
        if ((threadIdx.x & 31) == 0) dst[c] = dd_value(hh, ll);
    }
}

template <int NV>
__device__ __forceinline__ void warp_sums_to(double (&v)[NV], double* dst /* [NV] of this warp */)
{
#pragma unroll
    for (int k = 0; k < NV; k++) {
        double x = v[k];
#pragma unroll
        for (int off = 16; off >= 1; off >>= 1) x += __shfl_xor_sync(FULLMASK, x, off);
        if ((threadIdx.x & 31) == 0) dst[k] = x;
    }
}

// One problem per CTA: its trial's reduction, line-search step, L-BFGS
// update and next trial point.  Three passes over the problem's vectors;
// sums are per-warp partials in shared memory added in warp order (fixed
// order: results do not depend on scheduling).  The iterate, gradients and
// direction are FP64; the stored pairs (s_k, y_k) and the products with
// them are in double-float (see dd_fma); the scalar recursion is FP64.
__global__ void __launch_bounds__(BT) k_bstep(const BStepArgs A)
{
    if (!A.bc->go) return;
    const int k = blockIdx.x;
    if (!A.pactive[k]) return;
    constexpr int NB = NBASE + NPAIR * MAX_LBFGS_M;
    __shared__ double wpart[BW][NB];  // per warp: base dots, then NPAIR per slot
    __shared__ double red[NB];
    __shared__ double SYs[MAX_LBFGS_M * MAX_LBFGS_M], YYs[MAX_LBFGS_M * MAX_LBFGS_M];
    __shared__ double coef[2 * MAX_LBFGS_M + 2];  // cy[], cs[], cG, t
    __shared__ float2 coefp[2 * MAX_LBFGS_M];     // cy[], cs[] as float pairs
    __shared__ int act, fin;
    __shared__ unsigned shm[2 * BW];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const BProb p = A.P[k];
    BState* S = A.S + k;
    const int N = p.m + p.n, M = A.M;
    // the problem's vectors: distinct arrays (restrict: loads of a later
    // element may be issued before the stores of an earlier one)
    double* __restrict__ x = A.x + p.voff;
    double* __restrict__ G = A.G + p.voff;
    double* __restrict__ d = A.d + p.voff;
    double* __restrict__ xt = A.xt + p.voff;
    double* __restrict__ Gt = A.Gt + p.voff;
    unsigned long long* __restrict__ rowfx = A.rowfx;  // read in step 1, zeroed in step 5
    unsigned long long* __restrict__ colfx = A.colfx;
    const double* __restrict__ asorted = A.a_sorted;
    const double* __restrict__ bv_ = A.b;
    const FxScale fx = A.pfx[k];

    // 1. D, Gt = -grad D, Gt.d and ||Gt||_inf at the trial point
    {
        double v[4] = {0.0, 0.0, 0.0, 0.0};  // alpha.a + beta.b, Gt.d, (unused), ||.||_inf
#pragma unroll 4
        for (int e = threadIdx.x; e < N; e += BT) {
            double g, wt;
            if (e < p.m) {
                const int r = p.roff + e;
                wt = asorted[r];
                g = wt - (double)(long long)rowfx[r] * fx.from_r;
            } else {
                const int c = p.coff + (e - p.m);
                wt = bv_[c];
                g = wt - (double)(long long)colfx[c] * fx.from_c;
            }
            Gt[e] = -g;
            v[0] += xt[e] * wt;
            v[1] += -g * d[e];
            v[3] = fmax(v[3], fabs(g));
        }
#pragma unroll
        for (int off = 16; off >= 1; off >>= 1) v[3] = fmax(v[3], __shfl_xor_sync(FULLMASK, v[3], off));
        double sv[2] = {v[0], v[1]};
        warp_sums_to<2>(sv, wpart[w]);
        if (lane == 0) wpart[w][3] = v[3];
    }
    __syncthreads();
    // 2. the line search (or the start of the solve), one thread
    if (threadIdx.x == 0) {
        double ab = 0.0, dphi = 0.0, inf = 0.0;
        for (int q = 0; q < BW; q++) {
            ab += wpart[q][0];
            dphi += wpart[q][1];
            inf = fmax(inf, wpart[q][3]);
        }
        const double psi = psi_from_fx((long long)A.psix[2 * k], (long long)A.psix[2 * k + 1], fx.from_p);
        const double D = (A.kerr && *(volatile const int*)A.kerr) ? __longlong_as_double(0x7ff8000000000000ll)
                                                                  : ab - psi;
        const double F = -D;
        S->evals++;
        int a = ACT_RETRY, done = 0, status = OTGS_ENOTCONV;
        if (S->phase == PH_START) {
            S->F = F;
            S->ginf = inf;
            S->phase = PH_LS;
            a = ACT_START;
            if (inf <= A.tol || reached(S, D, A.rtol)) { done = 1; status = OTGS_OK; }
            else if (A.maxit <= 0) done = 1;
        } else {
            const int r = ls_update(S, F, dphi);
            if (r < 0) {
                done = 1;
                status = OTGS_ELINESEARCH;
            } else if (r > 0) {
                a = ACT_ACCEPT;
                S->F = F;
                S->ginf = inf;
                S->iter++;
                if (inf <= A.tol || reached(S, D, A.rtol) || stalled(S->F0, F, A.ftol)) {
                    done = 1;
                    status = OTGS_OK;
                }
                else if (S->iter >= A.maxit) done = 1;
            }
        }
        if (done) {
            S->done = 1;
            S->status = status;
            S->t_done_ms = (double)(b_gtimer() - A.bc->t_begin) * 1e-6;
            A.pactive[k] = 0;
            atomicSub(&A.bc->nactive, 1);
        }
        act = a;
        fin = done;
        coef[2 * MAX_LBFGS_M + 1] = S->t;
        coef[2 * MAX_LBFGS_M] = (double)S->head;
    }
    __syncthreads();
    const int a = act;
    if (a == ACT_ACCEPT || a == ACT_START) {
        // 3. accept: s = xt - x, y = Gt - G into the head slot, x = xt, G = Gt,
        // with the base dots and the NPAIR dots of every stored slot
        const int head = (int)coef[2 * MAX_LBFGS_M];
        float2* __restrict__ s_new = A.Sv + (int64_t)head * A.Ntot + p.voff;
        float2* __restrict__ y_new = A.Yv + (int64_t)head * A.Ntot + p.voff;
        float2* __restrict__ gp = A.Gp + p.voff;
        {
            double bv[NBASE] = {0.0, 0.0, 0.0, 0.0};
#pragma unroll 4
            for (int e = threadIdx.x; e < N; e += BT) {
                const double g = Gt[e];
                if (a == ACT_ACCEPT) {
                    const double sv = xt[e] - x[e], yv = g - G[e];
                    s_new[e] = dsplit(sv);
                    y_new[e] = dsplit(yv);
                    bv[DOT_SY] += sv * yv;
                    bv[DOT_SS] += sv * sv;
                    bv[DOT_YY] += yv * yv;
                }
                x[e] = xt[e];
                G[e] = g;
                gp[e] = dsplit(g);
                bv[DOT_GG] += g * g;
            }
            warp_sums_to<NBASE>(bv, wpart[w]);
        }
        const bool need_dir = !fin;
        // the pair dots: by enough warps that each lane sums at least two
        // entries (on small problems the warp trees of 2 x 20 floats cost
        // more than the entries)
        const int nwd = min(BW, max(1, (N + 63) / 64));
        if (need_dir && a == ACT_ACCEPT && w < nwd) {
            for (int q0 = 0; q0 < M; q0 += SLOT_GROUP) {
                float ph[SLOT_GROUP * NPAIR], pl[SLOT_GROUP * NPAIR];
#pragma unroll
                for (int c = 0; c < SLOT_GROUP * NPAIR; c++) ph[c] = pl[c] = 0.f;
                const float2* __restrict__ Sb = A.Sv + (int64_t)q0 * A.Ntot + p.voff;
                const float2* __restrict__ Yb = A.Yv + (int64_t)q0 * A.Ntot + p.voff;
#pragma unroll 2
                for (int e = threadIdx.x; e < N; e += nwd * 32) {
                    const float2 sn = s_new[e], yn = y_new[e], g = gp[e];
#pragma unroll
                    for (int u = 0; u < SLOT_GROUP; u++) {
                        if (q0 + u >= M) break;
                        const float2 sk = Sb[(int64_t)u * A.Ntot + e];
                        const float2 yk = Yb[(int64_t)u * A.Ntot + e];
                        dd_fma(sn, yk, ph[u * NPAIR + PD_SNEW_Y], pl[u * NPAIR + PD_SNEW_Y]);
                        dd_fma(sk, yn, ph[u * NPAIR + PD_S_YNEW], pl[u * NPAIR + PD_S_YNEW]);
                        dd_fma(yn, yk, ph[u * NPAIR + PD_YNEW_Y], pl[u * NPAIR + PD_YNEW_Y]);
                        dd_fma(g, sk, ph[u * NPAIR + PD_G_S], pl[u * NPAIR + PD_G_S]);
                        dd_fma(g, yk, ph[u * NPAIR + PD_G_Y], pl[u * NPAIR + PD_G_Y]);
                    }
                }
                warp_dd_sums_to<SLOT_GROUP * NPAIR>(ph, pl, wpart[w] + NBASE + q0 * NPAIR);
            }
        }
        if (need_dir)
            for (int q = threadIdx.x; q < M * M; q += BT) {
                SYs[q] = S->SY[q];
                YYs[q] = S->YY[q];
            }
        __syncthreads();
        if (!need_dir) return;  // (uniform)
        // the totals over warps, in warp order
        const int nv = NBASE + (a == ACT_ACCEPT ? NPAIR * M : 0);
        for (int c = threadIdx.x; c < NBASE + NPAIR * MAX_LBFGS_M; c += BT) {
            double t = 0.0;
            if (c < nv) {
                const int nq = c < NBASE ? BW : nwd;
                for (int q = 0; q < nq; q++) t += wpart[q][c];
            }
            red[c] = t;
        }
        __syncthreads();
        // 4. the direction (one warp)
        if (w == 0) {
            lbfgs_direction(S, SYs, YYs, red, reinterpret_cast<const double(*)[NPAIR]>(red + NBASE), M,
                            a == ACT_START, lane);
            static_assert(MAX_LBFGS_M <= 32, "one lane per history slot");
            if (lane < MAX_LBFGS_M) {
                const double cy = S->cy[lane], cs = S->cs[lane];
                coef[lane] = cy;
                coef[MAX_LBFGS_M + lane] = cs;
                coefp[lane] = dsplit(cy);
                coefp[MAX_LBFGS_M + lane] = dsplit(cs);
            }
            if (lane == 0) {
                coef[2 * MAX_LBFGS_M] = S->cG;
                coef[2 * MAX_LBFGS_M + 1] = S->t;
            }
        }
        __syncthreads();
    } else if (fin) {
        return;
    }
    // 5. (new direction d = cG G + sum_q cy_q y_q + cs_q s_q), the next trial
    // point xt = x + t d and its preparation
    const double t = coef[2 * MAX_LBFGS_M + 1];
    const bool newdir = a != ACT_RETRY;
    const double cG = coef[2 * MAX_LBFGS_M];
    float apos = 0.f, bpos = 0.f;
    const float2* __restrict__ Sb = A.Sv + p.voff;
    const float2* __restrict__ Yb = A.Yv + p.voff;
#pragma unroll 2
    for (int e = threadIdx.x; e < N; e += BT) {
        double dv;
        if (newdir) {
            float h = 0.f, l = 0.f;
            for (int q = 0; q < M; q++) {
                if (coef[q] != 0.0) dd_fma(coefp[q], Yb[(int64_t)q * A.Ntot + e], h, l);
                if (coef[MAX_LBFGS_M + q] != 0.0) dd_fma(coefp[MAX_LBFGS_M + q], Sb[(int64_t)q * A.Ntot + e], h, l);
            }
            dv = fma(cG, G[e], dd_value(h, l));
            d[e] = dv;
        } else {
            dv = d[e];
        }
        const double vv = fma(t, dv, x[e]);
        xt[e] = vv;
        if (e < p.m) {
            apos = fmaxf(apos, prep_row(vv, A.rowA + p.roff + e));
            rowfx[p.roff + e] = 0ull;
        } else {
            bpos = fmaxf(bpos, prep_col(true, vv, A.B2 + p.bcoff + (e - p.m)));
            colfx[p.coff + (e - p.m)] = 0ull;
        }
    }
    if (threadIdx.x < 2) A.psix[2 * k + threadIdx.x] = 0ull;  // read in step 1 (before the syncs since)
    store_scale(apos, bpos, k, p, A.gamma, A.pfx, shm);
}

__global__ void k_bcollect(const BState* S, BResult* R, int nprob)
{
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= nprob) return;
    const BState& s = S[k];
    BResult r;
    r.status = s.done ? s.status : OTGS_ENOTCONV;
    r.iter = s.iter;
    r.evals = s.evals;
    r.D = -s.F;
    r.ginf = s.ginf;
    r.t_ms = s.t_done_ms;
    R[k] = r;
}

// Caller layout <-> solver layout (per problem: sorted rows, then columns).
__global__ void k_bscatter(const BProb* __restrict__ P, const int32_t* __restrict__ perm, double* alpha,
                           double* beta, double* x, int to_solver)
{
    const BProb p = P[blockIdx.x];
    double* xv = x + p.voff;
    for (int e = threadIdx.x; e < p.m + p.n; e += blockDim.x) {
        if (e < p.m) {
            const int r = p.roff + e;
            if (to_solver) xv[e] = alpha[perm[r]];
            else alpha[perm[r]] = xv[e];
        } else {
            const int c = p.coff + (e - p.m);
            if (to_solver) xv[e] = beta[c];
            else beta[c] = xv[e];
        }
    }
}

// ------------------------------------------------------- shift search
// D(alpha + k 1, beta) is concave in k with derivative 1' grad_alpha D =
// sum a - sum T: per problem, a bracket [lo, hi] of the maximiser (from
// [-1/16, 1/16]) is grown (doubling) until the derivative is > 0 at lo and
// < 0 at hi, then halved.
struct ShiftState {
    double lo, hi, x;
    int lo_ok, hi_ok;
};

__global__ void __launch_bounds__(BT) k_shift_point(const BProb* __restrict__ P, ShiftState* S,
                                                    const double* __restrict__ alpha, double* work, int first)
{
    __shared__ double xs;
    const int k = blockIdx.x;
    const BProb p = P[k];
    if (threadIdx.x == 0) {
        ShiftState& s = S[k];
        if (first) {  // a start of the usual size: far points make every f positive (slow evaluations)
            s.lo = -0.0625;
            s.hi = 0.0625;
            s.lo_ok = 0;
            s.hi_ok = 0;
        }
        s.x = !s.hi_ok ? s.hi : (!s.lo_ok ? s.lo : 0.5 * (s.lo + s.hi));
        xs = s.x;
    }
    __syncthreads();
    for (int e = threadIdx.x; e < p.m; e += BT) work[p.roff + e] = alpha[p.roff + e] + xs;
}

__global__ void __launch_bounds__(BT) k_shift_update(const BProb* __restrict__ P, ShiftState* S,
                                                     const double* __restrict__ grad)
{
    __shared__ double sh[BW], tot[1];
    const int k = blockIdx.x;
    const BProb p = P[k];
    double v[1] = {0.0};
    for (int e = threadIdx.x; e < p.m; e += BT) v[0] += grad[p.roff + e];  // caller layout: rows of k contiguous
    cta_sum<1>(v, sh, tot);
    if (threadIdx.x != 0) return;
    ShiftState& s = S[k];
    const bool up = v[0] > 0.0;  // the maximiser lies above x
    if (!s.hi_ok) {
        if (up) { s.lo = s.hi; s.lo_ok = 1; s.hi *= 2.0; }
        else s.hi_ok = 1;
    } else if (!s.lo_ok) {
        if (!up) { s.hi = s.lo; s.lo *= 2.0; }
        else s.lo_ok = 1;
    } else if (up) {
        s.lo = s.x;
    } else {
        s.hi = s.x;
    }
}

__global__ void __launch_bounds__(BT) k_shift_apply(const BProb* __restrict__ P, const ShiftState* S, double* alpha)
{
    const BProb p = P[blockIdx.x];
    const ShiftState s = S[blockIdx.x];
    const double x = (s.lo_ok && s.hi_ok) ? 0.5 * (s.lo + s.hi) : s.x;
    for (int e = threadIdx.x; e < p.m; e += BT) alpha[p.roff + e] += x;
}

// ----------------------------------------------------------------- host
static bool batch_init(Handle* h)
{
    if (h->batch) return true;
    Batch* B = new (std::nothrow) Batch();
    if (!B) return h->fail(OTGS_ENOMEM, "batch allocation");
    h->batch = B;
    B->h = h;
    B->nprob = h->nprob;
    B->M = h->prm.lbfgs_m;
    B->Ntot = h->m + h->n;
    auto al = [&](size_t bytes, const char* w) { return h->dalloc(bytes, w); };
    B->S = (BState*)al(sizeof(BState) * (size_t)B->nprob, "batch states");
    B->bc = (BCtl*)al(sizeof(BCtl), "batch control");
    B->pactive = (int*)al(sizeof(int) * (size_t)B->nprob, "active problems");
    B->res = (BResult*)al(sizeof(BResult) * (size_t)B->nprob, "batch results");
    const size_t vb = sizeof(double) * (size_t)B->Ntot;
    B->x = (double*)al(vb, "x");
    B->G = (double*)al(vb, "G");
    B->d = (double*)al(vb, "d");
    B->xt = (double*)al(vb, "xt");
    B->Gt = (double*)al(vb, "Gt");
    B->Sv = (float2*)al(vb * B->M, "S");  // 8 bytes per entry: a float pair
    B->Yv = (float2*)al(vb * B->M, "Y");
    B->Gp = (float2*)al(vb, "G pairs");
    if (!B->S || !B->bc || !B->pactive || !B->res || !B->x || !B->G || !B->d || !B->xt || !B->Gt || !B->Sv ||
        !B->Yv || !B->Gp)
        return false;
    if (!h->ck(cudaMallocHost(&B->hbc, 2 * sizeof(BCtl)), "cudaMallocHost")) {
        B->hbc = nullptr;
        return false;
    }
    if (!h->ck(cudaStreamCreateWithFlags(&B->bst, cudaStreamNonBlocking), "cudaStreamCreate")) return false;
    for (cudaEvent_t& e : B->ev)
        if (!h->ck(cudaEventCreateWithFlags(&e, cudaEventDisableTiming), "cudaEventCreate")) return false;
    cudaStream_t st = h->st;
    if (!h->ck(cudaMemsetAsync(B->x, 0, vb, st), "memset") || !h->ck(cudaMemsetAsync(B->d, 0, vb, st), "memset") ||
        !h->ck(cudaMemsetAsync(B->Sv, 0, vb * B->M, st), "memset") ||
        !h->ck(cudaMemsetAsync(B->Yv, 0, vb * B->M, st), "memset"))
        return false;
    return h->ck(cudaStreamSynchronize(st), "batch init");
}

static BStepArgs step_args(Handle* h, Batch* B, double tol, double rtol, int maxit)
{
    BStepArgs a;
    memset(&a, 0, sizeof(a));
    a.P = h->bprob;
    a.S = B->S;
    a.bc = B->bc;
    a.pactive = B->pactive;
    a.pfx = h->pfx;
    a.gamma = (float)h->prm.gamma;
    a.rowfx = h->rowfx;
    a.colfx = h->colfx;
    a.psix = h->psix;
    a.kerr = h->kerr;
    a.a_sorted = h->a_sorted;
    a.b = h->b;
    a.x = B->x; a.G = B->G; a.d = B->d; a.xt = B->xt; a.Gt = B->Gt; a.Sv = B->Sv; a.Yv = B->Yv; a.Gp = B->Gp;
    a.Ntot = B->Ntot;
    a.M = B->M;
    a.rowA = h->rowA;
    a.B2 = h->B2;
    a.tol = tol;
    a.rtol = rtol;
    a.ftol = h->prm.ftol;
    a.maxit = maxit;
    return a;
}

// The trials of one graph launch.
static bool enqueue_trials(Handle* h, Batch* B, const BStepArgs& sa, int trials, cudaStream_t st)
{
    EvalArgs e = h->eval_args(nullptr, nullptr, false);
    e.psix = h->psix;  // per problem (k_bstep reads them), even for a batch of one
    e.gate = &B->bc->go;
    e.prob_active = B->pactive;
    e.pfx = h->pfx;
    const int n_ctas = std::min(CTAS_PER_SM * h->n_sm, h->hp.nitems());
    for (int q = 0; q < trials; q++) {
        k_bgate<<<1, 1, 0, st>>>(B->bc, h->ctl);
        launch_stream(e, n_ctas, st);
        launch_split_finish(e, st);
        launch_exact(e, h->n_sm, st);
        k_bstep<<<B->nprob, BT, 0, st>>>(sa);
    }
    return h->ck(cudaGetLastError(), "batch trial launch");
}

static bool capture_graph(Handle* h, Batch* B, double tol, double rtol, int maxit)
{
    // the captured arguments hold gamma and mu (theta, 1 / (2 gamma), the
    // fixed-point bounds), so a change of either needs a new graph
    if (B->gexec && B->g_plan == h->plan_gen && B->g_tol == tol && B->g_rtol == rtol &&
        B->g_maxit == maxit && B->g_ftol == h->prm.ftol && B->g_gamma == h->prm.gamma && B->g_mu == h->prm.mu)
        return true;
    if (B->gexec) {
        cudaGraphExecDestroy(B->gexec);
        B->gexec = nullptr;
    }
    const BStepArgs sa = step_args(h, B, tol, rtol, maxit);
    cudaGraph_t g = nullptr;
    if (!h->ck(cudaStreamBeginCapture(B->bst, cudaStreamCaptureModeThreadLocal), "cudaStreamBeginCapture"))
        return false;
    const bool ok = enqueue_trials(h, B, sa, TRIALS_PER_GRAPH, B->bst);
    const cudaError_t ce = cudaStreamEndCapture(B->bst, &g);
    if (!ok) {
        if (g) cudaGraphDestroy(g);
        return false;
    }
    if (!h->ck(ce, "cudaStreamEndCapture")) return false;
    const cudaError_t ie = cudaGraphInstantiate(&B->gexec, g, 0);
    cudaGraphDestroy(g);
    if (!h->ck(ie, "cudaGraphInstantiate")) {
        B->gexec = nullptr;
        return false;
    }
    B->g_plan = h->plan_gen;
    B->g_tol = tol;
    B->g_rtol = rtol;
    B->g_maxit = maxit;
    B->g_ftol = h->prm.ftol;
    B->g_gamma = h->prm.gamma;
    B->g_mu = h->prm.mu;
    return true;
}

static int batch_solve(Handle* h, double tol, int maxit, const double* target_host, double rtol)
{
    if (!batch_init(h)) return h->last_code;
    Batch* B = h->batch;
    if (B->M != h->prm.lbfgs_m) {
        h->fail(OTGS_EINVAL, "lbfgs_m changed after the first batch solve");
        return OTGS_EINVAL;
    }
    cudaStream_t st = B->bst;
    // the solve follows the work already queued on the handle's stream
    if (!h->ck(cudaEventRecord(B->ev[2], h->st), "cudaEventRecord") ||
        !h->ck(cudaStreamWaitEvent(st, B->ev[2], 0), "cudaStreamWaitEvent"))
        return h->last_code;
    double* dtarget = nullptr;
    if (target_host) {
        dtarget = B->Gt;  // scratch until the first evaluation overwrites it
        if (!h->ck(cudaMemcpyAsync(dtarget, target_host, sizeof(double) * B->nprob, cudaMemcpyHostToDevice, st),
                   "target H2D"))
            return h->last_code;
    }
    BCtl c0;
    memset(&c0, 0, sizeof(c0));
    c0.nactive = B->nprob;
    if (!h->ck(cudaMemcpyAsync(B->bc, &c0, sizeof(c0), cudaMemcpyHostToDevice, st), "control H2D")) return h->last_code;
    if (!h->ck(cudaMemsetAsync(h->kerr, 0, sizeof(int) * 4, st), "memset err")) return h->last_code;
    k_binit<<<B->nprob, BT, 0, st>>>(h->bprob, B->S, B->pactive, B->x, B->xt, h->rowA, h->B2, h->rowfx, h->colfx,
                                     h->pfx, (float)h->prm.gamma, B->M, dtarget, h->psix);
    k_bbegin<<<1, 1, 0, st>>>(B->bc);
    if (!h->ck(cudaGetLastError(), "batch start")) return h->last_code;
    if (!capture_graph(h, B, tol, rtol, maxit)) return h->last_code;
    // two graph launches in flight: the host reads one's count of running
    // problems while the next runs
    const long long max_launches = ((long long)maxit * (LS_MAX_EVALS + 2) + 16) / TRIALS_PER_GRAPH + 2;
    long long launched = 0;
    auto launch = [&](int slot) {
        if (!h->ck(cudaGraphLaunch(B->gexec, st), "cudaGraphLaunch")) return false;
        if (!h->ck(cudaMemcpyAsync(&B->hbc[slot], B->bc, sizeof(BCtl), cudaMemcpyDeviceToHost, st), "control D2H"))
            return false;
        if (!h->ck(cudaEventRecord(B->ev[slot], st), "cudaEventRecord")) return false;
        launched++;
        return true;
    };
    if (!launch(0) || !launch(1)) return h->last_code;
    for (long long i = 0;; i++) {
        const int slot = (int)(i & 1);
        if (!h->ck(cudaEventSynchronize(B->ev[slot]), "batch sync")) return h->last_code;
        if (B->hbc[slot].nactive == 0) break;
        if (launched >= max_launches) {  // the device loop always ends first; this is a second guard
            h->fail(OTGS_ENOTCONV, "batched solver exceeded its trial budget");
            return OTGS_ENOTCONV;
        }
        if (!launch(slot)) return h->last_code;
    }
    k_bcollect<<<(B->nprob + 127) / 128, 128, 0, st>>>(B->S, B->res, B->nprob);
    if (!h->ck(cudaStreamSynchronize(st), "batch sync")) return h->last_code;
    // the handle's stream sees the results
    if (!h->ck(cudaEventRecord(B->ev[2], st), "cudaEventRecord") ||
        !h->ck(cudaStreamWaitEvent(h->st, B->ev[2], 0), "cudaStreamWaitEvent"))
        return h->last_code;
    std::vector<BResult> r(B->nprob);
    if (!h->ck(cudaMemcpy(r.data(), B->res, sizeof(BResult) * r.size(), cudaMemcpyDeviceToHost), "results D2H"))
        return h->last_code;
    long long ev = 0;
    int worst = OTGS_OK;
    for (const BResult& x : r) {
        ev += x.evals;
        if (x.status != OTGS_OK && worst == OTGS_OK) worst = x.status;
    }
    h->stats_host.evals += ev;
    return worst;
}

}  // namespace otgs

using namespace otgs;

extern "C" {

int ot_gs_create_batch(ot_gs** out, int32_t nprob, const float* const* C, const int64_t* ldc, const double* const* a,
                       const double* const* b, const int32_t* const* labels, const int64_t* m, const int64_t* n,
                       const int32_t* L, double gamma, double mu, void* stream)
{
    set_create_error("");
    auto bad = [](const std::string& msg) {
        set_create_error(msg);
        return OTGS_EINVAL;
    };
    if (!out) return bad("h is NULL");
    *out = nullptr;
    if (nprob <= 0) return bad("need nprob > 0");
    if (!C || !ldc || !a || !b || !labels || !m || !n || !L) return bad("NULL array");
    for (int32_t k = 0; k < nprob; k++) {
        if (!C[k] || !a[k] || !b[k] || !labels[k]) return bad("NULL input pointer (problem " + std::to_string(k) + ")");
        if (m[k] <= 0 || n[k] <= 0 || L[k] <= 0 || ldc[k] < n[k])
            return bad("need m, n, L > 0 and ldc >= n (problem " + std::to_string(k) + ")");
    }
    if (!(gamma > 0.0) || !std::isfinite(gamma) || !(mu >= 0.0) || !std::isfinite(mu))
        return bad("need gamma > 0 and mu >= 0, finite");
    Handle* h = new (std::nothrow) Handle();
    if (!h) {
        set_create_error("out of host memory");
        return OTGS_ENOMEM;
    }
    if (!h->init(nprob, C, ldc, a, b, labels, m, n, L, gamma, mu, (cudaStream_t)stream)) {
        set_create_error(h->err);
        const int code = h->last_code ? h->last_code : OTGS_ECUDA;
        delete h;
        return code;
    }
    *out = reinterpret_cast<ot_gs*>(h);
    return OTGS_OK;
}

int ot_gs_batch_size(const ot_gs* hh, int32_t* nprob, int64_t* m_total, int64_t* n_total)
{
    if (!hh) return OTGS_EINVAL;
    const Handle* h = reinterpret_cast<const Handle*>(hh);
    if (nprob) *nprob = h->nprob;
    if (m_total) *m_total = h->m;
    if (n_total) *n_total = h->n;
    return OTGS_OK;
}

int ot_gs_batch_grad(ot_gs* hh, const double* alpha, const double* beta, double* D, double* grad)
{
    if (!hh) return OTGS_EINVAL;
    Handle* h = reinterpret_cast<Handle*>(hh);
    if (!alpha || !beta || !D) { h->fail(OTGS_EINVAL, "NULL pointer"); return OTGS_EINVAL; }
    return h->eval_batch(alpha, beta, D, grad) ? OTGS_OK : h->last_code;
}

int ot_gs_batch_solve(ot_gs* hh, double tol, int32_t maxit, const double* target_D, double target_rtol)
{
    if (!hh) return OTGS_EINVAL;
    Handle* h = reinterpret_cast<Handle*>(hh);
    if (!(tol >= 0.0) || maxit < 0 || (target_D && !(target_rtol >= 0.0))) {
        h->fail(OTGS_EINVAL, "need tol >= 0, maxit >= 0 and target_rtol >= 0");
        return OTGS_EINVAL;
    }
    return batch_solve(h, tol, maxit, target_D, target_D ? target_rtol : 0.0);
}

int ot_gs_batch_shift(ot_gs* hh, double* alpha, const double* beta, int32_t iters)
{
    if (!hh) return OTGS_EINVAL;
    Handle* h = reinterpret_cast<Handle*>(hh);
    if (!alpha || !beta || iters < 1 || iters > 200) {
        h->fail(OTGS_EINVAL, "need alpha, beta and 1 <= iters <= 200");
        return OTGS_EINVAL;
    }
    cudaStream_t st = h->st;
    ShiftState* S = (ShiftState*)h->dalloc(sizeof(ShiftState) * (size_t)h->nprob, "shift search");
    double* work = (double*)h->dalloc(sizeof(double) * (size_t)(2 * h->m + h->n) + sizeof(double) * h->nprob,
                                      "shift search");
    if (!S || !work) return h->last_code;
    double* grad = work + h->m;
    double* D = grad + h->m + h->n;
    // (alpha is in the caller's layout: the rows of problem k are entries [roff_k, roff_k + m_k))
    for (int it = 0; it < iters; it++) {
        k_shift_point<<<h->nprob, BT, 0, st>>>(h->bprob, S, alpha, work, it == 0);
        if (!h->eval_batch(work, beta, D, grad)) return h->last_code;
        k_shift_update<<<h->nprob, BT, 0, st>>>(h->bprob, S, grad);
    }
    k_shift_apply<<<h->nprob, BT, 0, st>>>(h->bprob, S, alpha);
    if (!h->ck(cudaStreamSynchronize(st), "shift search")) return OTGS_ECUDA;
    // the scratch goes back (allocated per call: this runs once per warm start)
    for (void* q : {(void*)S, (void*)work}) {
        for (size_t i = 0; i < h->allocs.size(); i++)
            if (h->allocs[i] == q) {
                h->allocs.erase(h->allocs.begin() + (long)i);
                break;
            }
        cudaFree(q);
    }
    return OTGS_OK;
}

int ot_gs_batch_set_state(ot_gs* hh, const double* alpha, const double* beta)
{
    if (!hh) return OTGS_EINVAL;
    Handle* h = reinterpret_cast<Handle*>(hh);
    if (!alpha || !beta) { h->fail(OTGS_EINVAL, "NULL pointer"); return OTGS_EINVAL; }
    if (!batch_init(h)) return h->last_code;
    k_bscatter<<<h->nprob, BT, 0, h->st>>>(h->bprob, h->dp.perm, const_cast<double*>(alpha),
                                           const_cast<double*>(beta), h->batch->x, 1);
    return h->ck(cudaGetLastError(), "batch set_state") ? OTGS_OK : OTGS_ECUDA;
}

int ot_gs_batch_result(ot_gs* hh, double* alpha, double* beta, double* D, double* grad_inf, int32_t* iters,
                       int32_t* status, int64_t* evals, double* t_ms)
{
    if (!hh) return OTGS_EINVAL;
    Handle* h = reinterpret_cast<Handle*>(hh);
    Batch* B = h->batch;
    if (!B) { h->fail(OTGS_EINVAL, "no batch solve yet"); return OTGS_EINVAL; }
    if (alpha && beta) {
        k_bscatter<<<h->nprob, BT, 0, h->st>>>(h->bprob, h->dp.perm, alpha, beta, B->x, 0);
        if (!h->ck(cudaGetLastError(), "batch result")) return OTGS_ECUDA;
    } else if (alpha || beta) {
        h->fail(OTGS_EINVAL, "alpha and beta go together");
        return OTGS_EINVAL;
    }
    std::vector<BResult> r(B->nprob);
    if (!h->ck(cudaMemcpyAsync(r.data(), B->res, sizeof(BResult) * r.size(), cudaMemcpyDeviceToHost, h->st), "D2H") ||
        !h->ck(cudaStreamSynchronize(h->st), "sync"))
        return OTGS_ECUDA;
    for (int k = 0; k < B->nprob; k++) {
        if (D) D[k] = r[k].D;
        if (grad_inf) grad_inf[k] = r[k].ginf;
        if (iters) iters[k] = r[k].iter;
        if (status) status[k] = r[k].status;
        if (evals) evals[k] = r[k].evals;
        if (t_ms) t_ms[k] = r[k].t_ms;
    }
    return OTGS_OK;
}

}  // extern "C"
