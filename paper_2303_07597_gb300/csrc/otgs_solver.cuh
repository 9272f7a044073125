// otgs_solver.cuh -- device L-BFGS state and the host side of the solve.
#pragma once

#include "otgs_handle.cuh"

namespace otgs {

constexpr int MAX_LBFGS_M = 32;
constexpr int SOLVER_THREADS = 256;
constexpr int TRACE_CAP = 1 << 16;  // objective trace entries kept per solve
constexpr int TRIALS_PER_SYNC = 16;  // line-search trials queued between host checks
// line search (same constants as the oracle)
constexpr double LS_C1 = 1e-4;
constexpr double LS_C2 = 0.9;
constexpr double LS_EPS_F = 1e-12;
constexpr int LS_MAX_EVALS = 40;
// pair-independent dot products
enum { DOT_SY = 0, DOT_SS, DOT_YY, DOT_GG, NBASE };
// per stored slot k: s_new.y_k, s_k.y_new, y_new.y_k, G.s_k, G.y_k
enum { PD_SNEW_Y = 0, PD_S_YNEW, PD_YNEW_Y, PD_G_S, PD_G_Y, NPAIR };

struct SolverState {
    int status, done, iter, npairs, head, accepted, refresh, force_accept;
    int ls_evals, have_hi, M, r, screening, maxit;
    int go;  // the current trial runs (set by the trial gate: not done, no refresh pending)
    int iter0;  // accepted iterations before this solve (a solve resumed from a saved state)
    int nan_eval;  // test hook: > 0, evaluations from this count on read D = NaN (0: off)
    long long evals;
    double tol, t, lo, Flo, dlo, hi, Fhi, dhi;
    double F, F0, dphi0, ginf, cG, budget_ns, ftol;
    unsigned long long t_start;
    unsigned long long t_begin;  // globaltimer when the solve was launched
    double* trace;               // [trace_cap][3]: D, ms since t_begin, evaluations
    int trace_cap;
    int pad_trace;
    double SY[MAX_LBFGS_M * MAX_LBFGS_M];  // SY[i*M + k] = s_i . y_k
    double YY[MAX_LBFGS_M * MAX_LBFGS_M];
    double cy[MAX_LBFGS_M], cs[MAX_LBFGS_M];
};

// ------------------------------------------------ device steps of L-BFGS
// Shared by the single-problem solver (SolverState) and the batched one (one
// state per problem): any St with the fields used below.

__device__ __forceinline__ double bracket_step(double lo, double Flo, double dlo, double hi, double Fhi, double dhi)
{
    const double w = hi - lo;
    double t = lo + 0.5 * w;
    if (dlo < 0.0 && dhi > 0.0) {
        t = lo - dlo * w / (dhi - dlo);
    } else {
        const double den = 2.0 * (Fhi - Flo - dlo * w);
        if (den > 0.0) t = lo - dlo * w * w / den;
    }
    if (!(t >= lo + 0.1 * w && t <= hi - 0.1 * w)) t = lo + 0.5 * w;
    return t;
}

// Objective stagnation: the accepted step lowered F = -D by at most
// ftol max(|F0|, |F|) (ftol = 0: never).
__device__ __forceinline__ bool stalled(double F0, double F, double ftol)
{
    return ftol > 0.0 && F0 - F <= ftol * fmax(fabs(F0), fabs(F));
}

// One trial of the strong-Wolfe line search on F = -D at step t with slope
// dphi = G(x + t d).d: 1 = accept, 0 = S->t holds the next trial, -1 = no
// acceptable step.
template <class St>
__device__ __forceinline__ int ls_update(St* S, double F, double dphi)
{
    const double F0 = S->F0, d0 = S->dphi0, t = S->t;
    const bool suff = (F <= F0 + LS_C1 * t * d0) || (F - F0 <= LS_EPS_F * fabs(F0) && dphi <= (2.0 * LS_C1 - 1.0) * d0);
    S->ls_evals++;
    if (S->force_accept || (suff && fabs(dphi) <= -LS_C2 * d0)) {
        S->force_accept = 0;
        return 1;
    }
    if (!suff || dphi >= 0.0) {
        S->hi = t; S->Fhi = F; S->dhi = dphi; S->have_hi = 1;
    } else {
        S->lo = t; S->Flo = F; S->dlo = dphi;
    }
    if (S->ls_evals >= LS_MAX_EVALS || (S->have_hi && S->hi - S->lo <= 1e-15 * S->hi)) {
        if (S->lo > 0.0) {  // evaluate once more at the last sufficient-decrease step and take it
            S->t = S->lo;
            S->force_accept = 1;
            return 0;
        }
        return -1;
    }
    S->t = S->have_hi ? bracket_step(S->lo, S->Flo, S->dlo, S->hi, S->Fhi, S->dhi) : 2.0 * t;
    return 0;
}

// One warp (all 32 lanes): keeps the new pair (slot S->head) when its
// curvature is positive enough (unless start), then the two-loop recursion
// (Nocedal & Wright, Alg. 7.4) on scalars, the descent check and the start of
// the next line search.  SY, YY: the M x M curvature matrices (shared memory
// copies of S->SY, S->YY, whose changed rows and columns are written back);
// base: s.y, s.s, y.y, G.G; pd[k]: the NPAIR dots of slot k.
//
// Lane u holds the u-th stored pair (oldest first).  The first loop, a_u =
// (s_u . G - sum_{v > u} a_v s_u . y_v) / s_u . y_u newest first, runs on
// lane 0 over shared-memory copies (each a_u needs every newer one, in that
// order).  The second, b_u = (h0 (y_u . G - sum_v a_v y_u . y_v) + sum_{v <
// u} (a_v - b_v) s_v . y_u) / s_u . y_u oldest first, is a triangular solve:
// every lane forms its first sum at once, and as each b_u is found it is
// broadcast and the lanes still waiting add their term.  The operations and
// their order are those of the textbook recursion term by term, so the
// result does not depend on how the work is spread over the lanes.
template <class St>
__device__ void lbfgs_direction(St* S, double* SY, double* YY, const double* base, const double (*pd)[NPAIR], int M,
                                bool start, int lane)
{
    int np = S->npairs, hd = S->head;
    if (!start) {
        const int head = hd;
        const double sy = base[DOT_SY];
        if (sy > 1e-12 * sqrt(base[DOT_SS] * base[DOT_YY])) {
            if (lane < M) {
                SY[head * M + lane] = pd[lane][PD_SNEW_Y];  // s_head . y_k
                SY[lane * M + head] = pd[lane][PD_S_YNEW];  // s_k . y_head
                YY[head * M + lane] = pd[lane][PD_YNEW_Y];
                YY[lane * M + head] = pd[lane][PD_YNEW_Y];
            }
            __syncwarp();
            if (lane == 0) {
                SY[head * M + head] = sy;
                YY[head * M + head] = base[DOT_YY];
            }
            __syncwarp();
            if (lane < M) {
                S->SY[head * M + lane] = SY[head * M + lane];
                S->SY[lane * M + head] = SY[lane * M + head];
                S->YY[head * M + lane] = YY[head * M + lane];
                S->YY[lane * M + head] = YY[lane * M + head];
            }
            hd = (head + 1) % M;
            if (np < M) np++;
        } else if (np == M) {
            np = M - 1;  // the rejected pair overwrote the oldest slot
        }
    }
    const bool mine = lane < np;
    const int i = mine ? ((hd - np + lane) % M + M) % M : 0;  // this lane's slot
    __shared__ double a_s[MAX_LBFGS_M];
    __shared__ int idx_s[MAX_LBFGS_M];
    if (mine) idx_s[lane] = i;
    __syncwarp();
    // first loop, newest to oldest (lane 0)
    if (lane == 0)
        for (int u = np - 1; u >= 0; u--) {
            const int iu = idx_s[u];
            double sq = pd[iu][PD_G_S];
            for (int v = u + 1; v < np; v++) sq -= a_s[v] * SY[iu * M + idx_s[v]];
            a_s[u] = sq / SY[iu * M + iu];
        }
    __syncwarp();
    const double a = mine ? a_s[lane] : 0.0;
    double h0 = 1.0;
    if (np > 0) {
        const int nw = ((hd - 1) % M + M) % M;
        h0 = SY[nw * M + nw] / YY[nw * M + nw];
    }
    // second loop, oldest to newest
    double yq = mine ? pd[i][PD_G_Y] : 0.0;
    for (int v = 0; v < np; v++) {
        const double av = __shfl_sync(0xffffffffu, a, v);
        const int iv = __shfl_sync(0xffffffffu, i, v);
        if (mine) yq -= av * YY[i * M + iv];
    }
    double yr = h0 * yq, b = 0.0;
    for (int u = 0; u < np; u++) {
        if (lane == u) b = yr / SY[i * M + i];
        const double cu = __shfl_sync(0xffffffffu, a - b, u);
        const int iu = __shfl_sync(0xffffffffu, i, u);
        if (mine && lane > u) yr += cu * SY[iu * M + i];
    }
    // d = -(h0 q + sum (a - b) s) = -h0 G + h0 sum a y - sum (a - b) s
    double cG = -h0;
    double dphi0 = cG * base[DOT_GG];
    const double cy = h0 * a, cs = -(a - b);
    for (int u = 0; u < np; u++) {  // every lane, the same sum in the same order
        const double cyu = __shfl_sync(0xffffffffu, cy, u), csu = __shfl_sync(0xffffffffu, cs, u);
        const int iu = __shfl_sync(0xffffffffu, i, u);
        dphi0 += cyu * pd[iu][PD_G_Y] + csu * pd[iu][PD_G_S];
    }
    const bool descent = dphi0 < 0.0;
    if (!descent) {  // not a descent direction: restart from -G
        np = 0;
        cG = -1.0;
        dphi0 = -base[DOT_GG];
    }
    // slot k's coefficients: from the lane that holds slot k, 0 for slots not stored
    const int uk = ((lane - hd + np) % M + M) % M;  // the position slot k = lane would have
    const bool held = descent && lane < M && uk < np;
    const double cyk = __shfl_sync(0xffffffffu, cy, held ? uk : 0);
    const double csk = __shfl_sync(0xffffffffu, cs, held ? uk : 0);
    if (lane < MAX_LBFGS_M) {
        S->cy[lane] = held ? cyk : 0.0;
        S->cs[lane] = held ? csk : 0.0;
    }
    if (lane == 0) {
        S->head = hd;
        S->npairs = np;
        S->cG = cG;
        S->dphi0 = dphi0;
        S->F0 = S->F;
        const double ginf = S->ginf;
        S->t = (S->iter == 0 && np == 0 && ginf > 0.0) ? 1.0 / ginf : 1.0;
        S->lo = 0.0; S->Flo = S->F; S->dlo = dphi0;
        S->hi = 0.0; S->Fhi = 0.0; S->dhi = 0.0; S->have_hi = 0;
        S->ls_evals = 0;
        S->force_accept = 0;
    }
    __syncwarp();
}

struct Solver {
    Handle* h = nullptr;
    int N = 0, M = 0, nblk = 0;
    SolverState* state = nullptr;
    SolverState* hstate = nullptr;  // pinned
    double *x = nullptr, *G = nullptr, *d = nullptr, *xt = nullptr, *Gt = nullptr;
    double *Sv = nullptr, *Yv = nullptr;
    double *pbase = nullptr, *ppair = nullptr;  // dot partials
    double* trace = nullptr;                    // objective trace of the last solve
    int trace_len = 0;
    double D = 0.0, ginf = 0.0;
    int iters = 0;
    ~Solver();
    bool init(Handle* h);
    int run(double tol, int maxit);
    bool resume = false;  // the next run continues the state restored by ot_gs_restore_state
    long long evals0 = 0; // evaluations of the restored state
    bool eval_trial();
    void launch_dots(bool start);
};

}  // namespace otgs
