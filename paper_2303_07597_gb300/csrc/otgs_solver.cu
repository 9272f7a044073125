// otgs_solver.cu -- L-BFGS on -D (Eq. 4) with a strong-Wolfe line search,
// all state and arithmetic on the device (FP64).
//
// The two-loop recursion (Nocedal & Wright, Alg. 7.4) only needs dot products
// of the current gradient G with the stored pairs and of the pairs with each
// other.  Those come from one multi-dot pass per accepted step; the scalar
// recursion then runs on one warp and one more pass forms the direction
//   d = cG G + sum_k cy_k y_k + sum_k cs_k s_k.
// The line search is a state machine in one thread: it reads D and the slope
// of the trial evaluation, and sets the next trial step, or accepts.  Alg. 1's
// snapshot refresh (with the rebuild of N) runs every r accepted iterations.
#include <algorithm>
#include <cmath>
#include <cstddef>
#include <cstring>

#include "otgs_solver.cuh"

namespace otgs {

#define FULLMASK 0xffffffffu

// ------------------------------------------------------------------ kernels
// x_t = x + t d; also the preparation of x_t for the evaluation kernel (the
// same per-row and per-column records as the plain preparation kernel).
__global__ void k_trial(SolverState* S, const double* __restrict__ x, const double* __restrict__ d, double* xt,
                        float4* rowA, float2* B2, double* alpha_eval, unsigned long long* rowfx,
                        unsigned long long* colfx, EvalCtl* ctl, int m, int n, int npad)
{
    if (!S->go) return;  // the same for every thread
    const double t = S->t;
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    float apos = 0.f, bpos = 0.f;
    if (i < m) {
        const double v = fma(t, d[i], x[i]);
        xt[i] = v;
        alpha_eval[i] = v;
        apos = prep_row(v, rowA + i);
        rowfx[i] = 0ull;
    }
    if (i < npad) {
        double v = 0.0;
        if (i < n) {
            v = fma(t, d[m + i], x[m + i]);
            xt[m + i] = v;
            colfx[i] = 0ull;
        }
        bpos = prep_col(i < n, v, B2 + i);
    }
    record_max(ctl, apos, bpos);
}

__device__ __forceinline__ unsigned long long gtimer()
{
    unsigned long long t;
    asm volatile("mov.u64 %0, %globaltimer;" : "=l"(t));
    return t;
}

// Entry iter of the objective trace: D = -F, device time since the launch of
// the solve, evaluations so far.
__device__ __forceinline__ void trace_put(SolverState* S, double F)
{
    const int k = S->iter - S->iter0;
    if (!S->trace || k >= S->trace_cap) return;
    double* e = S->trace + 3 * (size_t)k;
    e[0] = -F;
    e[1] = (double)(gtimer() - S->t_begin) * 1e-6;
    e[2] = (double)S->evals;
}

// Line-search state machine (same rule as the oracle): scal = {D, Gt.d, ||Gt||_inf}.
__global__ void k_linesearch(SolverState* S, const double* scal)
{
    if (!S->go) return;
    S->evals++;
    S->accepted = 0;
    S->refresh = 0;
    const double F = (S->nan_eval > 0 && S->evals >= S->nan_eval) ? __longlong_as_double(0x7ff8000000000000ll)
                                                                    : -scal[0];
    const double dphi = scal[1];
    const int r = ls_update(S, F, dphi);
    if (r < 0) {
        S->status = OTGS_ELINESEARCH;
        S->done = 1;
    } else if (r > 0) {
        S->accepted = 1;
        S->F = F;
        S->ginf = scal[2];
        S->iter++;
        trace_put(S, F);
        if (S->ginf <= S->tol || stalled(S->F0, F, S->ftol)) {
            S->status = OTGS_OK;
            S->done = 1;
        } else if (S->iter >= S->maxit) {
            S->status = OTGS_ENOTCONV;
            S->done = 1;
        } else if (S->budget_ns > 0.0 && (double)(gtimer() - S->t_start) > S->budget_ns) {
            S->status = OTGS_ETIMEOUT;
            S->done = 1;
        }
        S->refresh = S->screening && !S->done && (S->iter % S->r == 0);
    }
}

// Fixed-order block sum of NV values (one per thread) into out[0..NV).
template <int NV>
__device__ __forceinline__ void block_sum(double (&acc)[NV], double* out)
{
    __shared__ double sh[SOLVER_THREADS / 32][NV];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
#pragma unroll
    for (int k = 0; k < NV; k++) {
        double v = acc[k];
        for (int off = 16; off >= 1; off >>= 1) v += __shfl_xor_sync(FULLMASK, v, off);
        if (lane == 0) sh[w][k] = v;
    }
    __syncthreads();
    if (threadIdx.x < NV) {
        double v = 0.0;
        for (int q = 0; q < SOLVER_THREADS / 32; q++) v += sh[q][threadIdx.x];
        out[threadIdx.x] = v;
    }
}

// Accept: s = xt - x, y = Gt - G into slot head; x = xt, G = Gt; the
// pair-independent dots s.y, s.s, y.y, G.G per block.
__global__ void __launch_bounds__(SOLVER_THREADS) k_accept(SolverState* S, double* x, double* G, const double* xt,
                                                          const double* Gt, double* Sv, double* Yv, int N,
                                                          double* pbase)
{
    if (!S->go || !S->accepted) return;
    const int head = S->head;
    double* s_new = Sv + (size_t)head * N;
    double* y_new = Yv + (size_t)head * N;
    double acc[NBASE] = {0.0, 0.0, 0.0, 0.0};
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < N; i += gridDim.x * blockDim.x) {
        const double s = xt[i] - x[i], y = Gt[i] - G[i], g = Gt[i];
        s_new[i] = s;
        y_new[i] = y;
        x[i] = xt[i];
        G[i] = g;
        acc[DOT_SY] += s * y;
        acc[DOT_SS] += s * s;
        acc[DOT_YY] += y * y;
        acc[DOT_GG] += g * g;
    }
    block_sum<NBASE>(acc, pbase + (size_t)blockIdx.x * NBASE);
}

// G.G at the start of a solve (no pairs yet).
__global__ void __launch_bounds__(SOLVER_THREADS) k_gg(const double* G, int N, double* pbase)
{
    double acc[NBASE] = {0.0, 0.0, 0.0, 0.0};
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < N; i += gridDim.x * blockDim.x) acc[DOT_GG] += G[i] * G[i];
    block_sum<NBASE>(acc, pbase + (size_t)blockIdx.x * NBASE);
}

// Per stored slot k = blockIdx.y: s_new.y_k, s_k.y_new, y_new.y_k, G.s_k, G.y_k.
__global__ void __launch_bounds__(SOLVER_THREADS) k_pairdots(const SolverState* S, const double* G, const double* Sv,
                                                            const double* Yv, int N, double* ppair)
{
    if (!S->go || !S->accepted) return;
    const int k = blockIdx.y, head = S->head;
    const double* s_new = Sv + (size_t)head * N;
    const double* y_new = Yv + (size_t)head * N;
    const double* sk = Sv + (size_t)k * N;
    const double* yk = Yv + (size_t)k * N;
    double acc[NPAIR] = {0.0, 0.0, 0.0, 0.0, 0.0};
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < N; i += gridDim.x * blockDim.x) {
        const double sn = s_new[i], yn = y_new[i], g = G[i], s = sk[i], y = yk[i];
        acc[PD_SNEW_Y] += sn * y;
        acc[PD_S_YNEW] += s * yn;
        acc[PD_YNEW_Y] += yn * y;
        acc[PD_G_S] += g * s;
        acc[PD_G_Y] += g * y;
    }
    block_sum<NPAIR>(acc, ppair + ((size_t)k * gridDim.x + blockIdx.x) * NPAIR);
}

// Sum block partials in block order; then (one warp) the two-loop recursion
// on scalars, the descent check, and the start of the next line search.  It
// also runs after the iteration that ends a solve, so that the state a solve
// stops in is the one an unfinished solve goes on from (a saved state then
// resumes exactly).
__global__ void __launch_bounds__(SOLVER_THREADS) k_direction(SolverState* S, const double* pbase, const double* ppair,
                                                             int nblocks, int start)
{
    if (start ? S->done : (!S->go || !S->accepted)) return;
    const int M = S->M;
    __shared__ double base[NBASE];
    __shared__ double pd[MAX_LBFGS_M][NPAIR];
    // the curvature matrices, so that the serial recursion below reads shared memory
    __shared__ double SY[MAX_LBFGS_M * MAX_LBFGS_M], YY[MAX_LBFGS_M * MAX_LBFGS_M];
    for (int q = threadIdx.x; q < M * M; q += blockDim.x) {
        SY[q] = S->SY[q];
        YY[q] = S->YY[q];
    }
    // one warp per quantity: lane-strided partial sums, then a fixed xor tree
    const int lane = threadIdx.x & 31, nwarps = blockDim.x >> 5;
    for (int q = threadIdx.x >> 5; q < NBASE + M * NPAIR; q += nwarps) {
        double v = 0.0;
        if (q < NBASE) {
            for (int b = lane; b < nblocks; b += 32) v += pbase[(size_t)b * NBASE + q];
        } else if (!start) {
            const int k = (q - NBASE) / NPAIR, c = (q - NBASE) % NPAIR;
            for (int b = lane; b < nblocks; b += 32) v += ppair[((size_t)k * nblocks + b) * NPAIR + c];
        }
#pragma unroll
        for (int off = 16; off >= 1; off >>= 1) v += __shfl_xor_sync(FULLMASK, v, off);
        if (lane == 0) {
            if (q < NBASE) base[q] = v;
            else pd[(q - NBASE) / NPAIR][(q - NBASE) % NPAIR] = v;
        }
    }
    __syncthreads();
    if (threadIdx.x >= 32) return;
    lbfgs_direction(S, SY, YY, base, pd, M, start != 0, lane);
}

// d = cG G + sum_k cy_k y_k + sum_k cs_k s_k
__global__ void k_combine(const SolverState* S, const double* G, const double* Sv, const double* Yv, double* d,
                          int N, int M, int start)
{
    if (start ? S->done : (!S->go || !S->accepted)) return;
    const double cG = S->cG;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < N; i += gridDim.x * blockDim.x) {
        double v = cG * G[i];
        for (int k = 0; k < M; k++) {
            const double cy = S->cy[k], cs = S->cs[k];
            if (cy != 0.0) v += cy * Yv[(size_t)k * N + i];
            if (cs != 0.0) v += cs * Sv[(size_t)k * N + i];
        }
        d[i] = v;
    }
}

// Start of a solve: F, ||G|| from the evaluation at x; convergence at x.
__global__ void k_start(SolverState* S, const double* scal)
{
    S->F = -scal[0];
    S->ginf = scal[2];
    S->evals++;
    if (!isfinite(S->F) || !isfinite(S->ginf)) {  // a non-finite start point (or a failed evaluation)
        S->status = OTGS_ENONFINITE;
        S->done = 1;
    } else if (S->ginf <= S->tol) {
        S->status = OTGS_OK;
        S->done = 1;
    } else if (S->maxit <= 0) {
        S->status = OTGS_ENOTCONV;
        S->done = 1;
    }
    S->t_start = gtimer();
    trace_put(S, S->F);
}

__global__ void k_begin(SolverState* S) { S->t_begin = gtimer(); }

// Continues a restored state: the stopping rule of this solve, its trace
// (entry 0 = the restored iterate), and Alg. 1's snapshot refresh that an
// unfinished solve would take after the restored iteration.
__global__ void k_resume(SolverState* S, double tol, int maxit, double budget_ns, double ftol, double* trace,
                         int trace_cap, int r, int screening)
{
    S->tol = tol;
    S->maxit = maxit;
    S->budget_ns = budget_ns;
    S->ftol = ftol;
    S->trace = trace;
    S->trace_cap = trace_cap;
    S->r = r;
    S->screening = screening;
    S->iter0 = S->iter;
    S->status = OTGS_ENOTCONV;
    S->done = 0;
    S->go = 0;
    S->accepted = 0;
    S->refresh = screening && S->iter > 0 && S->iter % r == 0;
    if (S->iter >= maxit) S->done = 1;
    S->t_start = gtimer();
    trace_put(S, S->F);
}

// Opens a line-search trial: it runs only while the solve is not done and no
// snapshot refresh is waiting for the host.  A running trial starts with a
// cleared evaluation control word (and screening maxima).
__global__ void k_gate(SolverState* S, EvalCtl* ctl, unsigned* gmax)
{
    const int go = !S->done && !S->refresh;
    S->go = go;
    if (!go) return;
    ctl_clear(ctl);
    if (gmax)
        for (int k = 0; k < 4; k++) gmax[k] = 0u;
}

__global__ void k_clear_refresh(SolverState* S) { S->refresh = 0; }

// ------------------------------------------------------------------- host
bool Solver::init(Handle* h_)
{
    h = h_;
    N = (int)(h->m + h->n);
    M = h->prm.lbfgs_m;
    // blocks of the vector kernels: enough to cover N once (up to two per SM)
    nblk = (int)std::min<int64_t>(2 * std::max(1, h->n_sm), (N + SOLVER_THREADS - 1) / SOLVER_THREADS);
    auto al = [&](size_t bytes, const char* w) { return h->dalloc(bytes, w); };
    state = (SolverState*)al(sizeof(SolverState), "solver state");
    x = (double*)al(sizeof(double) * N, "x");
    G = (double*)al(sizeof(double) * N, "G");
    d = (double*)al(sizeof(double) * N, "d");
    xt = (double*)al(sizeof(double) * N, "xt");
    Gt = (double*)al(sizeof(double) * N, "Gt");
    Sv = (double*)al(sizeof(double) * (size_t)N * M, "S");
    Yv = (double*)al(sizeof(double) * (size_t)N * M, "Y");
    pbase = (double*)al(sizeof(double) * (size_t)nblk * NBASE, "dot partials");
    ppair = (double*)al(sizeof(double) * (size_t)nblk * M * NPAIR, "pair dot partials");
    trace = (double*)al(sizeof(double) * 3 * (size_t)TRACE_CAP, "objective trace");
    if (cudaMallocHost(&hstate, sizeof(SolverState)) != cudaSuccess) {
        hstate = nullptr;
        return h->fail(OTGS_ENOMEM, "cudaMallocHost(solver state)");
    }
    if (!state || !x || !G || !d || !xt || !Gt || !Sv || !Yv || !pbase || !ppair || !trace) return false;
    cudaMemsetAsync(x, 0, sizeof(double) * N, h->st);
    cudaMemsetAsync(Sv, 0, sizeof(double) * (size_t)N * M, h->st);
    cudaMemsetAsync(Yv, 0, sizeof(double) * (size_t)N * M, h->st);
    return h->ck(cudaGetLastError(), "solver init");
}

Solver::~Solver()
{
    if (hstate) cudaFreeHost(hstate);
}

int Solver::run(double tol, int maxit)
{
    cudaStream_t st = h->st;
    SolverState init;
    memset(&init, 0, sizeof(init));
    init.tol = tol;
    init.maxit = maxit;
    init.M = M;
    init.r = h->prm.r;
    init.screening = h->prm.use_screening;
    init.budget_ns = h->prm.time_budget_ms > 0 ? h->prm.time_budget_ms * 1e6 : 0.0;
    init.ftol = h->prm.ftol;
    init.npairs = 0;
    init.head = 0;
    init.status = OTGS_ENOTCONV;
    init.trace = trace;
    init.trace_cap = TRACE_CAP;
    init.nan_eval = (int)std::min<int64_t>(std::max<int64_t>(h->dbg_nan_eval, 0), INT32_MAX);
    trace_len = 0;
    const bool resumed = resume;
    resume = false;
    if (resumed) {
        if (h->prm.use_screening && !h->snap_valid) {
            h->fail(OTGS_EINVAL, "the restored state has no snapshot: resume with use_screening = 0");
            return OTGS_EINVAL;
        }
        k_begin<<<1, 1, 0, st>>>(state);
        k_resume<<<1, 1, 0, st>>>(state, tol, maxit, init.budget_ns, init.ftol, trace, TRACE_CAP, h->prm.r,
                                  h->prm.use_screening);
    } else {
        if (!h->ck(cudaMemcpyAsync(state, &init, sizeof(init), cudaMemcpyHostToDevice, st), "state H2D"))
            return h->last_code;
        k_begin<<<1, 1, 0, st>>>(state);
    }
    // as Alg. 1 starts: snapshot at the start point, N empty
    if (resumed) {
    } else if (h->prm.use_screening) {
        h->invalidate_screen();
        if (!h->ensure_screen()) return h->last_code;
        cudaMemsetAsync(h->Nmask, 0, sizeof(uint32_t) * (size_t)h->L * h->ntiles, st);
        h->snap_valid = true;  // replaced right away by the snapshot at x
        if (!h->snapshot_at(x, true, x + h->m, false, nullptr, G, nullptr)) return h->last_code;
    } else {
        if (!h->eval_dense(x, true, x + h->m, nullptr, G, nullptr, false)) return h->last_code;
    }
    if (!resumed) {
        k_start<<<1, 1, 0, st>>>(state, h->scal);
        k_gg<<<nblk, SOLVER_THREADS, 0, st>>>(G, N, pbase);
        k_direction<<<1, SOLVER_THREADS, 0, st>>>(state, pbase, ppair, nblk, 1);
        k_combine<<<nblk, SOLVER_THREADS, 0, st>>>(state, G, Sv, Yv, d, N, M, 1);
    }
    const int npad = padded_cols(h->n);
    const int tb = (std::max((int)h->m, npad) + 255) / 256;
    const size_t hdr = offsetof(SolverState, tol);  // the int fields and the eval counter
    const long long max_trials = (long long)maxit * (LS_MAX_EVALS + 2) + 16;
    // Trials are queued up to TRIALS_PER_SYNC at a time; each opens with k_gate, so
    // the ones queued after the solve ended, or after an iteration that asks
    // for a snapshot refresh (Alg. 1, every r accepted iterations), do
    // nothing.  The host then takes the snapshot at the accepted iterate and
    // queues more.
    h->eval_gate = &state->go;
    bool ok = true;
    while (ok) {
        if (!h->ck(cudaMemcpyAsync(hstate, state, hdr, cudaMemcpyDeviceToHost, st), "state D2H") ||
            !h->ck(cudaStreamSynchronize(st), "solver sync")) {
            ok = false;
            break;
        }
        if (hstate->done) break;
        if (hstate->refresh) {
            h->eval_gate = nullptr;
            ok = h->snapshot_at(x, true, x + h->m, true, nullptr, nullptr, nullptr);
            h->eval_gate = &state->go;
            k_clear_refresh<<<1, 1, 0, st>>>(state);
            if (!ok) break;
        }
        if (hstate->evals - 1 >= max_trials) {  // the device loop always ends first; this is a second guard
            h->fail(OTGS_ENOTCONV, "solver exceeded its trial budget");
            break;
        }
        // with screening, trials up to the next refresh (every r accepted
        // iterations, each taking at least one trial) and two more for line
        // searches that need a second one: the trials queued after the refresh
        // point only pass through the gate
        int nq = TRIALS_PER_SYNC;
        if (hstate->screening && hstate->r > 0)
            nq = std::min(nq, hstate->r - hstate->iter % hstate->r + 2);
        for (int q = 0; q < nq; q++) {
            k_gate<<<1, 1, 0, st>>>(state, h->ctl, h->prm.use_screening ? h->gmax : nullptr);
            k_trial<<<tb, 256, 0, st>>>(state, x, d, xt, h->rowA, h->B2, h->alpha_eval, h->rowfx, h->colfx,
                                        h->ctl, (int)h->m, (int)h->n, npad);
            if (!eval_trial()) { ok = false; break; }
            k_linesearch<<<1, 1, 0, st>>>(state, h->scal);
            k_accept<<<nblk, SOLVER_THREADS, 0, st>>>(state, x, G, xt, Gt, Sv, Yv, N, pbase);
            k_pairdots<<<dim3(nblk, M), SOLVER_THREADS, 0, st>>>(state, G, Sv, Yv, N, ppair);
            k_direction<<<1, SOLVER_THREADS, 0, st>>>(state, pbase, ppair, nblk, 0);
            k_combine<<<nblk, SOLVER_THREADS, 0, st>>>(state, G, Sv, Yv, d, N, M, 0);
        }
        if (ok && !h->ck(cudaGetLastError(), "solver launch")) ok = false;
    }
    h->eval_gate = nullptr;
    if (!ok) return h->last_code;
    if (!h->ck(cudaMemcpyAsync(hstate, state, sizeof(SolverState), cudaMemcpyDeviceToHost, st), "state D2H") ||
        !h->ck(cudaStreamSynchronize(st), "solver sync"))
        return h->last_code;
    h->stats_host.iters = hstate->iter;
    trace_len = std::min(hstate->iter - hstate->iter0 + 1, TRACE_CAP);
    // the trial evaluations (all but the first, counted when it was made)
    const long long trials = resumed ? hstate->evals - evals0 : hstate->evals - 1;
    if (trials > 0) {
        if (h->prm.use_screening) h->count_screened_evals(trials);
        else h->count_dense_evals(trials);
    }
    iters = hstate->iter;
    D = -hstate->F;
    ginf = hstate->ginf;
    return hstate->status;
}

// Evaluation of the trial point prepared by k_trial.
bool Solver::eval_trial()
{
    const double* beta = xt + h->m;
    if (h->prm.use_screening) return h->eval_screened_prepped(beta, Gt, d);
    return h->eval_dense_prepped(beta, Gt, d);
}

// ---------------------------------------------------------- saved states
// A saved solver state is one device buffer: a header, then the L-BFGS state
// (the struct, x, G, the direction, the stored pairs), then, when the handle
// holds a snapshot, Alg. 1's screening state (z~, o~, alpha~, beta~, N).
namespace {
constexpr uint64_t STATE_MAGIC = 0x5441545347544f31ull;
constexpr int32_t STATE_VERSION = 1;
struct StateHeader {
    uint64_t magic;
    int32_t version, M;
    int64_t m, n;
    int32_t L, ntiles;
    int32_t has_snap, pad;
    double gamma, mu;
    int64_t bytes;
};
struct StateLayout {
    size_t st, x, G, d, S, Y, zt, ot, as, bs, Nm, total;
};
inline size_t a16(size_t v) { return (v + 15) / 16 * 16; }
StateLayout state_layout(const Handle* h, int M, bool snap)
{
    const size_t N = (size_t)(h->m + h->n), lz = (size_t)h->L * h->ntiles * TW, lu = (size_t)h->L * h->ntiles;
    StateLayout o;
    size_t at = a16(sizeof(StateHeader));
    auto take = [&](size_t bytes) {
        const size_t p = at;
        at = a16(at + bytes);
        return p;
    };
    o.st = take(sizeof(SolverState));
    o.x = take(8 * N);
    o.G = take(8 * N);
    o.d = take(8 * N);
    o.S = take(8 * N * M);
    o.Y = take(8 * N * M);
    o.zt = o.ot = o.as = o.bs = o.Nm = 0;
    if (snap) {
        o.zt = take(4 * lz);
        o.ot = take(4 * lz);
        o.as = take(8 * (size_t)h->m);
        o.bs = take(8 * (size_t)h->n);
        o.Nm = take(4 * lu);
    }
    o.total = at;
    return o;
}
}  // namespace

}  // namespace otgs

using namespace otgs;

extern "C" {

int ot_gs_state_size(ot_gs* hh, int64_t* bytes)
{
    if (!hh || !bytes) return OTGS_EINVAL;
    Handle* h = reinterpret_cast<Handle*>(hh);
    if (!single_problem(h)) return OTGS_EINVAL;
    const int M = h->solver ? h->solver->M : h->prm.lbfgs_m;
    *bytes = (int64_t)state_layout(h, M, h->screen_alloc && h->snap_valid).total;
    return OTGS_OK;
}

int ot_gs_get_state(ot_gs* hh, void* dst, int64_t bytes)
{
    if (!hh) return OTGS_EINVAL;
    Handle* h = reinterpret_cast<Handle*>(hh);
    if (!single_problem(h)) return OTGS_EINVAL;
    if (!dst) { h->fail(OTGS_EINVAL, "NULL pointer"); return OTGS_EINVAL; }
    if (!h->solver) { h->fail(OTGS_EINVAL, "no solver state yet (solve or set_state first)"); return OTGS_EINVAL; }
    Solver* s = h->solver;
    const bool snap = h->screen_alloc && h->snap_valid;
    const StateLayout o = state_layout(h, s->M, snap);
    if (bytes < (int64_t)o.total) { h->fail(OTGS_EINVAL, "buffer smaller than ot_gs_state_size"); return OTGS_EINVAL; }
    StateHeader hd;
    memset(&hd, 0, sizeof(hd));
    hd.magic = STATE_MAGIC;
    hd.version = STATE_VERSION;
    hd.M = s->M;
    hd.m = h->m;
    hd.n = h->n;
    hd.L = h->L;
    hd.ntiles = h->ntiles;
    hd.has_snap = snap ? 1 : 0;
    hd.gamma = h->prm.gamma;
    hd.mu = h->prm.mu;
    hd.bytes = (int64_t)o.total;
    char* b = static_cast<char*>(dst);
    const size_t N = (size_t)(h->m + h->n), lz = (size_t)h->L * h->ntiles * TW, lu = (size_t)h->L * h->ntiles;
    cudaStream_t st = h->st;
    auto cp = [&](size_t off, const void* src, size_t n, cudaMemcpyKind k) {
        return h->ck(cudaMemcpyAsync(b + off, src, n, k, st), "state copy");
    };
    bool ok = cp(0, &hd, sizeof(hd), cudaMemcpyHostToDevice) &&
              cp(o.st, s->state, sizeof(SolverState), cudaMemcpyDeviceToDevice) &&
              cp(o.x, s->x, 8 * N, cudaMemcpyDeviceToDevice) && cp(o.G, s->G, 8 * N, cudaMemcpyDeviceToDevice) &&
              cp(o.d, s->d, 8 * N, cudaMemcpyDeviceToDevice) &&
              cp(o.S, s->Sv, 8 * N * s->M, cudaMemcpyDeviceToDevice) &&
              cp(o.Y, s->Yv, 8 * N * s->M, cudaMemcpyDeviceToDevice);
    if (ok && snap)
        ok = cp(o.zt, h->zt, 4 * lz, cudaMemcpyDeviceToDevice) && cp(o.ot, h->ot, 4 * lz, cudaMemcpyDeviceToDevice) &&
             cp(o.as, h->alpha_snap, 8 * (size_t)h->m, cudaMemcpyDeviceToDevice) &&
             cp(o.bs, h->beta_snap, 8 * (size_t)h->n, cudaMemcpyDeviceToDevice) &&
             cp(o.Nm, h->Nmask, 4 * lu, cudaMemcpyDeviceToDevice);
    if (!ok || !h->ck(cudaStreamSynchronize(st), "state sync")) return h->last_code;
    return OTGS_OK;
}

int ot_gs_restore_state(ot_gs* hh, const void* src, int64_t bytes)
{
    if (!hh) return OTGS_EINVAL;
    Handle* h = reinterpret_cast<Handle*>(hh);
    if (!single_problem(h)) return OTGS_EINVAL;
    if (!src || bytes < (int64_t)sizeof(StateHeader)) { h->fail(OTGS_EINVAL, "NULL or short state"); return OTGS_EINVAL; }
    StateHeader hd;
    if (!h->ck(cudaMemcpyAsync(&hd, src, sizeof(hd), cudaMemcpyDeviceToHost, h->st), "state header") ||
        !h->ck(cudaStreamSynchronize(h->st), "state sync"))
        return h->last_code;
    if (hd.magic != STATE_MAGIC || hd.version != STATE_VERSION) {
        h->fail(OTGS_EINVAL, "not a saved solver state");
        return OTGS_EINVAL;
    }
    if (hd.m != h->m || hd.n != h->n || hd.L != h->L || hd.ntiles != h->ntiles || hd.M != h->prm.lbfgs_m ||
        hd.gamma != h->prm.gamma || hd.mu != h->prm.mu) {
        h->fail(OTGS_EINVAL, "the saved state belongs to another problem (sizes, classes, lbfgs_m, gamma or mu)");
        return OTGS_EINVAL;
    }
    const StateLayout o = state_layout(h, hd.M, hd.has_snap != 0);
    if (hd.bytes != (int64_t)o.total || bytes < hd.bytes) { h->fail(OTGS_EINVAL, "state size mismatch"); return OTGS_EINVAL; }
    if (!h->solver) {
        h->solver = new (std::nothrow) Solver();
        if (!h->solver || !h->solver->init(h)) {
            delete h->solver;
            h->solver = nullptr;
            return h->last_code ? h->last_code : OTGS_ENOMEM;
        }
    }
    Solver* s = h->solver;
    if (s->M != hd.M) { h->fail(OTGS_EINVAL, "lbfgs_m changed after the first solve"); return OTGS_EINVAL; }
    const char* b = static_cast<const char*>(src);
    const size_t N = (size_t)(h->m + h->n), lz = (size_t)h->L * h->ntiles * TW, lu = (size_t)h->L * h->ntiles;
    cudaStream_t st = h->st;
    auto cp = [&](void* dst, size_t off, size_t n) {
        return h->ck(cudaMemcpyAsync(dst, b + off, n, cudaMemcpyDeviceToDevice, st), "state copy");
    };
    bool ok = cp(s->state, o.st, sizeof(SolverState)) && cp(s->x, o.x, 8 * N) && cp(s->G, o.G, 8 * N) &&
              cp(s->d, o.d, 8 * N) && cp(s->Sv, o.S, 8 * N * s->M) && cp(s->Yv, o.Y, 8 * N * s->M);
    if (!ok) return h->last_code;
    if (hd.has_snap) {
        if (!h->ensure_screen()) return h->last_code;
        ok = cp(h->zt, o.zt, 4 * lz) && cp(h->ot, o.ot, 4 * lz) && cp(h->alpha_snap, o.as, 8 * (size_t)h->m) &&
             cp(h->beta_snap, o.bs, 8 * (size_t)h->n) && cp(h->Nmask, o.Nm, 4 * lu) && h->zt_tiles();
        if (!ok) return h->last_code;
        h->snap_valid = true;
    } else {
        h->invalidate_screen();
    }
    if (!h->ck(cudaMemcpyAsync(s->hstate, s->state, sizeof(SolverState), cudaMemcpyDeviceToHost, st), "state D2H") ||
        !h->ck(cudaStreamSynchronize(st), "state sync"))
        return h->last_code;
    s->evals0 = s->hstate->evals;
    s->iters = s->hstate->iter;
    s->D = -s->hstate->F;
    s->ginf = s->hstate->ginf;
    s->resume = true;
    return OTGS_OK;
}

int ot_gs_solve(ot_gs* hh, double tol, int32_t maxit)
{
    if (!hh) return OTGS_EINVAL;
    Handle* h = reinterpret_cast<Handle*>(hh);
    if (!single_problem(h)) return OTGS_EINVAL;
    if (h->shard) {
        h->fail(OTGS_EINVAL, "a column shard's objective is partial: combine the shards' evaluations");
        return OTGS_EINVAL;
    }
    if (!(tol >= 0.0) || maxit < 0) { h->fail(OTGS_EINVAL, "need tol >= 0 and maxit >= 0"); return OTGS_EINVAL; }
    if (!h->solver) {
        h->solver = new (std::nothrow) Solver();
        if (!h->solver || !h->solver->init(h)) {
            delete h->solver;
            h->solver = nullptr;
            if (!h->last_code) h->fail(OTGS_ENOMEM, "solver allocation");
            return h->last_code;
        }
    } else if (h->solver->M != h->prm.lbfgs_m) {
        h->fail(OTGS_EINVAL, "lbfgs_m changed after the first solve");
        return OTGS_EINVAL;
    }
    return h->solver->run(tol, maxit);
}

int ot_gs_get_solution(ot_gs* hh, double* alpha, double* beta, double* D, double* grad_inf, int32_t* iters)
{
    if (!hh) return OTGS_EINVAL;
    Handle* h = reinterpret_cast<Handle*>(hh);
    if (!single_problem(h)) return OTGS_EINVAL;
    if (!h->solver) { h->fail(OTGS_EINVAL, "no solve yet"); return OTGS_EINVAL; }
    Solver* s = h->solver;
    if (alpha) launch_permute_f64(s->x, h->dp.perm, (int32_t)h->m, alpha, false, h->st);
    if (beta && !h->ck(cudaMemcpyAsync(beta, s->x + h->m, sizeof(double) * h->n, cudaMemcpyDeviceToDevice, h->st),
                       "copy"))
        return OTGS_ECUDA;
    if (!h->ck(cudaStreamSynchronize(h->st), "sync")) return OTGS_ECUDA;
    if (D) *D = s->D;
    if (grad_inf) *grad_inf = s->ginf;
    if (iters) *iters = s->iters;
    return OTGS_OK;
}

int ot_gs_get_trace(ot_gs* hh, double* D, double* t_ms, int64_t* evals, int32_t cap, int32_t* count)
{
    if (!hh) return OTGS_EINVAL;
    Handle* h = reinterpret_cast<Handle*>(hh);
    if (!h->solver) { h->fail(OTGS_EINVAL, "no solve yet"); return OTGS_EINVAL; }
    if (cap < 0 || (cap > 0 && (!D || !t_ms || !evals))) { h->fail(OTGS_EINVAL, "bad trace buffers"); return OTGS_EINVAL; }
    Solver* s = h->solver;
    const int k = std::min<int>(cap, s->trace_len);
    if (count) *count = s->trace_len;
    if (k == 0) return OTGS_OK;
    std::vector<double> buf(3 * (size_t)k);
    if (!h->ck(cudaMemcpyAsync(buf.data(), s->trace, sizeof(double) * buf.size(), cudaMemcpyDeviceToHost, h->st),
               "trace D2H") ||
        !h->ck(cudaStreamSynchronize(h->st), "sync"))
        return OTGS_ECUDA;
    for (int i = 0; i < k; i++) {
        D[i] = buf[3 * i];
        t_ms[i] = buf[3 * i + 1];
        evals[i] = (int64_t)buf[3 * i + 2];
    }
    return OTGS_OK;
}

int ot_gs_set_state(ot_gs* hh, const double* alpha, const double* beta)
{
    if (!hh) return OTGS_EINVAL;
    Handle* h = reinterpret_cast<Handle*>(hh);
    if (!single_problem(h)) return OTGS_EINVAL;
    if (!alpha || !beta) { h->fail(OTGS_EINVAL, "NULL pointer"); return OTGS_EINVAL; }
    if (!h->solver) {
        h->solver = new (std::nothrow) Solver();
        if (!h->solver || !h->solver->init(h)) {
            delete h->solver;
            h->solver = nullptr;
            return h->last_code ? h->last_code : OTGS_ENOMEM;
        }
    }
    Solver* s = h->solver;
    s->resume = false;
    launch_permute_f64(alpha, h->dp.perm, (int32_t)h->m, s->x, true, h->st);
    if (!h->ck(cudaMemcpyAsync(s->x + h->m, beta, sizeof(double) * h->n, cudaMemcpyDeviceToDevice, h->st), "copy"))
        return OTGS_ECUDA;
    h->invalidate_screen();
    return h->ck(cudaGetLastError(), "set_state") ? OTGS_OK : OTGS_ECUDA;
}

}  // extern "C"
